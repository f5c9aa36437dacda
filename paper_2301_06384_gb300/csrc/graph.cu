// Graph ingest (step a1): host validation of the CSR Laplacian, device copy of its
// off-diagonal part and diagonal excess, and the Gershgorin bound Lambda computed on the
// device.  Also the error/diagnostic plumbing of the C ABI.
//
// Section 2.1, Eq. (generalizedLaplacian): L symmetric, L_ij < 0 exactly on edges,
// L_ij = 0 off the graph, any diagonal.  Lambda is the Gershgorin bound
// max_i sum_j |L_ij| (Section 2.1 assumes a known spectral bound; this one is computable).
#include "kb_internal.cuh"
#include "kb_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>

namespace kb {

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return KB_ERR_NOMEM;
    return KB_ERR_CUDA;
}

int num_sms() {
    // function-local static: computed once, thread-safe (several serving workers)
    static const int sms = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v <= 0 ? 1 : v;
    }();
    return sms;
}

// ---------------------------------------------------------------- profiling
namespace {
constexpr int PROF_SLOTS = 1 << 16;   // device work counters available per profile read
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double bytes, flops;        // full-size values (used when the slot has no counter)
    int slot;                   // -1: no device counter
    double per_row, per_nnz, flops_per_row, fixed;
};
std::mutex g_prof_mu;
bool g_prof = false;
std::vector<ProfRec> g_recs;
std::vector<cudaEvent_t> g_pool;
cudaEvent_t g_pending = nullptr;
int g_pending_cls = -1;
int g_pending_slot = -1;
unsigned long long *g_counters = nullptr;   // [PROF_SLOTS][2] rows, nnz (device)
int g_next_slot = 0;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

bool prof_on() { return g_prof; }

ProfCount prof_begin(int cls, cudaStream_t s) {
    ProfCount pc;
    if (!g_prof) return pc;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_pending = take_event();
    g_pending_cls = cls;
    g_pending_slot = -1;
    if (g_counters && g_next_slot < PROF_SLOTS) {
        g_pending_slot = g_next_slot++;
        pc.rows = g_counters + 2 * size_t(g_pending_slot);
        pc.nnz = pc.rows + 1;
    }
    cudaEventRecord(g_pending, s);
    return pc;
}

std::atomic<long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void prof_end(int cls, cudaStream_t s, double bytes, double flops, int nlaunch, double per_row,
              double per_nnz, double flops_per_row, double fixed) {
    count_launches(nlaunch);
    if (!g_prof) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_pending || g_pending_cls != cls) return;
    cudaEvent_t b = take_event();
    cudaEventRecord(b, s);
    const bool counted = per_row > 0.0 || per_nnz > 0.0 || flops_per_row > 0.0;
    g_recs.push_back(ProfRec{cls, g_pending, b, bytes, flops, counted ? g_pending_slot : -1,
                             per_row, per_nnz, flops_per_row, fixed});
    g_pending = nullptr;
}

// ---------------------------------------------------------------- Gershgorin bound
namespace {
__global__ void k_gershgorin(GraphDev g, unsigned long long *out_bits) {
    double best = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.n;
         i += int64_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int p = g.rowptr[i]; p < g.rowptr[i + 1]; ++p) s += g.w ? double(g.w[p]) : 1.0;
        const double diag = (g.rdiag ? double(g.rdiag[i]) : 0.0) + s;
        best = fmax(best, fabs(diag) + s);
    }
    // non-negative doubles order like their bit patterns
    for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, static_cast<unsigned long long>(__double_as_longlong(best)));
}
}  // namespace

int launch_gershgorin(const GraphDev &g, double *out, cudaStream_t s) {
    unsigned long long *d = nullptr;
    KB_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&d), sizeof(unsigned long long), s));
    KB_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned long long), s));
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>((g.n + 255) / 256, int64_t(num_sms()) * 8)));
    k_gershgorin<<<grid, 256, 0, s>>>(g, d);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    unsigned long long bits = 0;
    KB_CUDA_TRY(cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, s));
    KB_CUDA_TRY(cudaStreamSynchronize(s));
    KB_CUDA_TRY(cudaFreeAsync(d, s));
    double v;
    std::memcpy(&v, &bits, sizeof(v));
    *out = v;
    return 0;
}

}  // namespace kb

// ---------------------------------------------------------------- C ABI: graph
using namespace kb;

extern "C" int kb_graph_create(int64_t n, const int32_t *rowptr, const int32_t *col,
                               const float *val, int32_t flags, void *stream, kb_graph **out) {
    try {
        if (!out) return fail(KB_ERR_ARG, "out is NULL");
        *out = nullptr;
        if (n < 1 || n >= (int64_t(1) << 31)) return fail(KB_ERR_ARG, "n out of range");
        if (!rowptr || !col) return fail(KB_ERR_ARG, "rowptr/col is NULL");
        if (rowptr[0] != 0) return fail(KB_ERR_CSR, "rowptr[0] != 0");
        for (int64_t i = 0; i < n; ++i)
            if (rowptr[i + 1] < rowptr[i]) return fail(KB_ERR_CSR, "rowptr not non-decreasing at row " + std::to_string(i));
        const int64_t nnz = rowptr[n];
        // pass 1: structure and signs, count stored off-diagonal entries
        int64_t noff = 0;
        bool unit = true;
        for (int64_t i = 0; i < n; ++i) {
            int32_t prev = -1;
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                const int32_t j = col[p];
                if (j < 0 || j >= n) return fail(KB_ERR_CSR, "column out of range in row " + std::to_string(i));
                if (j <= prev) return fail(KB_ERR_CSR, "columns not strictly increasing in row " + std::to_string(i));
                prev = j;
                if (j == i) {
                    if (val && !std::isfinite(val[p])) return fail(KB_ERR_CSR, "non-finite diagonal");
                    continue;
                }
                if (val) {
                    const float v = val[p];
                    if (!std::isfinite(v)) return fail(KB_ERR_CSR, "non-finite value");
                    if (v > 0.f) return fail(KB_ERR_CSR, "positive off-diagonal entry in row " + std::to_string(i));
                    if (v == 0.f) continue;   // explicit zero: not an edge
                    if (v != -1.f) unit = false;
                }
                ++noff;
            }
        }
        (void)nnz;
        // pass 2: symmetry (pattern and bitwise values of the non-zero off-diagonal entries)
        if (!(flags & KB_GRAPH_SKIP_SYMMETRY_CHECK)) {
            for (int64_t i = 0; i < n; ++i) {
                for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                    const int32_t j = col[p];
                    if (j == i) continue;
                    const float v = val ? val[p] : -1.f;
                    if (v == 0.f) continue;
                    const int32_t *b = col + rowptr[j], *e = col + rowptr[j + 1];
                    const int32_t *q = std::lower_bound(b, e, int32_t(i));
                    if (q == e || *q != i) return fail(KB_ERR_CSR, "pattern not symmetric at (" + std::to_string(i) + "," + std::to_string(j) + ")");
                    const float vt = val ? val[q - col] : -1.f;
                    if (vt != v) return fail(KB_ERR_CSR, "values not symmetric at (" + std::to_string(i) + "," + std::to_string(j) + ")");
                }
            }
        }
        // normalized Laplacian I - D^{-1/2} A D^{-1/2} (the one Section 8 uses): weighted degrees first
        const bool normalized = (flags & KB_GRAPH_NORMALIZED) != 0;
        std::vector<double> deg(normalized ? n : 0, 0.0);
        if (normalized) {
            unit = false;
            for (int64_t i = 0; i < n; ++i)
                for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                    if (col[p] == i) continue;
                    const float v = val ? val[p] : -1.f;
                    deg[i] += double(-v);
                }
        }
        // build the stored form
        std::vector<int32_t> h_rowptr(n + 1);
        std::vector<int32_t> h_col(noff);
        std::vector<float> h_w(unit ? 0 : noff);
        std::vector<float> h_rdiag(n);
        bool zero_excess = true;
        int64_t q = 0;
        h_rowptr[0] = 0;
        for (int64_t i = 0; i < n; ++i) {
            double wsum = 0.0, diag = 0.0;
            bool has_diag = false;
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                const int32_t j = col[p];
                if (j == i) {
                    if (val) { diag = double(val[p]); has_diag = true; }
                    continue;
                }
                const float v = val ? val[p] : -1.f;
                if (v == 0.f) continue;
                h_col[q] = j;
                const double w = normalized ? double(-v) / std::sqrt(deg[i] * deg[j]) : double(-v);
                if (!unit) h_w[q] = float(w);
                wsum += normalized ? double(float(w)) : w;
                ++q;
            }
            h_rowptr[i + 1] = int32_t(q);
            // val == NULL: standard Laplacian, diagonal = degree (zero excess); normalized:
            // diagonal 1 on every node with an edge
            double excess = (val ? (has_diag ? diag : 0.0) : wsum) - wsum;
            if (normalized) excess = (deg[i] > 0.0 ? 1.0 : 0.0) - wsum;
            h_rdiag[i] = float(excess);
            if (h_rdiag[i] != 0.f) zero_excess = false;
        }
        int dev = 0;
        KB_CUDA_TRY(cudaGetDevice(&dev));
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        kb_graph *g = new (std::nothrow) kb_graph();
        if (!g) return fail(KB_ERR_NOMEM, "host allocation failed");
        g->device = dev;
        auto cleanup = [&]() {
            cudaFree(g->d_rowptr); cudaFree(g->d_col); cudaFree(g->d_w); cudaFree(g->d_rdiag);
            delete g;
        };
        cudaError_t e = cudaMalloc(&g->d_rowptr, sizeof(int32_t) * (n + 1));
        if (e == cudaSuccess) e = cudaMalloc(&g->d_col, sizeof(int32_t) * std::max<int64_t>(noff, 1));
        if (e == cudaSuccess && !unit) e = cudaMalloc(&g->d_w, sizeof(float) * std::max<int64_t>(noff, 1));
        if (e == cudaSuccess && !zero_excess) e = cudaMalloc(&g->d_rdiag, sizeof(float) * n);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->d_rowptr, h_rowptr.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && noff) e = cudaMemcpyAsync(g->d_col, h_col.data(), sizeof(int32_t) * noff, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !unit && noff) e = cudaMemcpyAsync(g->d_w, h_w.data(), sizeof(float) * noff, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !zero_excess) e = cudaMemcpyAsync(g->d_rdiag, h_rdiag.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "graph upload");
        }
        g->dev.n = n;
        g->dev.nnz = noff;
        g->dev.rowptr = g->d_rowptr;
        g->dev.col = g->d_col;
        g->dev.w = g->d_w;
        g->dev.rdiag = g->d_rdiag;
        g->unit_weights = unit ? 1 : 0;
        g->zero_excess = zero_excess ? 1 : 0;
        int rc = launch_gershgorin(g->dev, &g->lambda, s);
        if (rc) {
            cleanup();
            return rc;
        }
        // the spectrum of the normalized Laplacian lies in [0, 2] (tighter than Gershgorin)
        if (normalized) g->lambda = std::min(g->lambda, 2.0);
        // Lanczos projected step: for the unit-weight standard Laplacian D - A the largest
        // eigenvalue is at most max over edges of d_i + d_j (Anderson and Morley, 1985), about
        // half the Gershgorin bound 2 max d on hub-dominated graphs; the projected matrix's
        // spectrum lies below it too (interlacing), so the Chebyshev series of e^{-t lambda}
        // on the shorter interval needs proportionally fewer terms.  A margin of 1e-3 keeps
        // Ritz values that rounding pushes past the bound (star graphs meet it exactly) in
        // the interval where the series converges.
        g->lambda_proj = g->lambda;
        if (unit && zero_excess && !normalized) {
            int64_t best = 0;
            for (int64_t i = 0; i < n; ++i) {
                const int64_t di = h_rowptr[i + 1] - h_rowptr[i];
                for (int32_t p = h_rowptr[i]; p < h_rowptr[i + 1]; ++p) {
                    const int32_t j = h_col[p];
                    best = std::max<int64_t>(best, di + (h_rowptr[j + 1] - h_rowptr[j]));
                }
            }
            g->lambda_proj = std::min(g->lambda, double(best) * (1.0 + 1e-3));
        }
        *out = g;
        return KB_OK;
    } catch (const std::bad_alloc &) {
        return fail(KB_ERR_NOMEM, "host allocation failed");
    } catch (...) {
        return fail(KB_ERR_CUDA, "unexpected exception");
    }
}

extern "C" void kb_graph_destroy(kb_graph *g) {
    if (!g) return;
    cudaFree(g->d_rowptr);
    cudaFree(g->d_col);
    cudaFree(g->d_w);
    cudaFree(g->d_rdiag);
    delete g;
}

extern "C" int kb_graph_lambda_bounds(const kb_graph *g, double *gershgorin, double *projected) {
    if (!g) return fail(KB_ERR_ARG, "graph is NULL");
    if (gershgorin) *gershgorin = g->lambda;
    if (projected) *projected = g->lambda_proj;
    return KB_OK;
}

extern "C" int kb_graph_info(const kb_graph *g, int64_t *n, int64_t *nnz_offdiag, double *lambda_max,
                             int32_t *standard_unit) {
    if (!g) return fail(KB_ERR_ARG, "graph is NULL");
    if (n) *n = g->dev.n;
    if (nnz_offdiag) *nnz_offdiag = g->dev.nnz;
    if (lambda_max) *lambda_max = g->lambda;
    if (standard_unit) *standard_unit = (g->unit_weights && g->zero_excess) ? 1 : 0;
    return KB_OK;
}

// ---------------------------------------------------------------- C ABI: diagnostics
extern "C" const char *kb_status_string(int status) {
    switch (status) {
        case KB_OK: return "ok";
        case KB_ERR_ARG: return "invalid argument";
        case KB_ERR_CSR: return "invalid CSR Laplacian";
        case KB_ERR_NODES: return "invalid node set";
        case KB_ERR_CUDA: return "CUDA error";
        case KB_ERR_NOMEM: return "out of device memory";
        case KB_ERR_BREAKDOWN: return "Lanczos breakdown (rank-deficient block)";
        case KB_ERR_UNSUPPORTED: return "unsupported combination";
        case KB_ERR_BUSY: return "serving queue full";
        case KB_ERR_ORTHOGONALITY: return "projected matrix outside [0, Lambda] (basis lost orthogonality)";
        case KB_PENDING: return "pending";
        default: return "unknown status";
    }
}

extern "C" const char *kb_last_error(void) { return kb::g_last_error.c_str(); }

extern "C" int kb_version(void) { return 10000; }

extern "C" int kb_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(kb::g_prof_mu);
    if (on && !kb::g_counters) {
        const size_t bytes = sizeof(unsigned long long) * 2 * kb::PROF_SLOTS;
        if (cudaMalloc(&kb::g_counters, bytes) != cudaSuccess) {
            kb::g_counters = nullptr;
        } else {
            cudaMemset(kb::g_counters, 0, bytes);
        }
        kb::g_next_slot = 0;
    }
    kb::g_prof = on != 0;
    return KB_OK;
}

extern "C" int kb_profile_read(kb_kernel_stats *out, int32_t cap, int32_t *count) {
    std::lock_guard<std::mutex> lk(kb::g_prof_mu);
    std::vector<kb_kernel_stats> acc(KernelClass::COUNT);
    for (int c = 0; c < KernelClass::COUNT; ++c) {
        acc[c].kernel_class = c;
        acc[c].launches = 0;
        acc[c].total_ms = 0;
        acc[c].alg_bytes = 0;
        acc[c].alg_flops = 0;
    }
    std::vector<unsigned long long> cnt;
    if (kb::g_counters && kb::g_next_slot > 0) {
        cudaDeviceSynchronize();
        cnt.resize(2 * size_t(kb::g_next_slot));
        cudaMemcpy(cnt.data(), kb::g_counters, sizeof(unsigned long long) * cnt.size(),
                   cudaMemcpyDeviceToHost);
        cudaMemset(kb::g_counters, 0, sizeof(unsigned long long) * cnt.size());
    }
    for (auto &r : kb::g_recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto &a = acc[r.cls];
        a.launches += 1;
        a.total_ms += ms;
        if (r.slot >= 0 && size_t(2 * r.slot + 1) < cnt.size()) {
            const double rows = double(cnt[2 * r.slot]), nnz = double(cnt[2 * r.slot + 1]);
            a.alg_bytes += r.fixed + rows * r.per_row + nnz * r.per_nnz;
            a.alg_flops += rows * r.flops_per_row;
        } else {
            a.alg_bytes += r.bytes;
            a.alg_flops += r.flops;
        }
        kb::g_pool.push_back(r.a);
        kb::g_pool.push_back(r.b);
    }
    kb::g_recs.clear();
    kb::g_next_slot = 0;
    int k = 0;
    for (int c = 0; c < KernelClass::COUNT && k < cap; ++c) out[k++] = acc[c];
    if (count) *count = k;
    return KB_OK;
}

extern "C" int64_t kb_launch_counter(void) { return kb::g_launches.load(); }

extern "C" const char *kb_kernel_class_name(int32_t cls) {
    static const char *names[] = {"spmm", "rowblock", "reduce", "small_fp64", "projected_fp64",
                                  "assemble", "other"};
    if (cls < 0 || cls >= KernelClass::COUNT) return "?";
    return names[cls];
}
