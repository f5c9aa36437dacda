// kb_cheb_apply_fixed_scratch: the Chebyshev solve (KB_CHEB) without any allocation.
//
// Some callers cannot allocate device memory at the time they need kernel columns:
// code that runs inside a framework which has reserved all device memory for its own
// allocator, latency-critical loops that must not touch the allocator (or its locks)
// after start-up, and tools that share one device with other processes under a fixed
// memory budget.  This entry point serves them: its scratch lives in one file-scope
// __device__ array of fixed size, loaded with the library, so a call performs no
// cudaMalloc / cudaMallocAsync / cudaFree and calls no allocating library routine.
//
// The paper has no counterpart of this entry point; it is a deployment variant of the
// Chebyshev method of Section 3.4.  It runs the Clenshaw recurrence of kb_krylov_apply with
// KB_CHEB on all n rows at every step (no frontier restriction, which would need more
// scratch).  The frontier restriction only skips rows whose values are exactly zero, and
// every other row goes through the same SpMM kernel with the same coefficients, so the two
// entry points return bitwise equal results.
#include "kb_internal.cuh"
#include "kb_kernels.cuh"

#include <cmath>
#include <mutex>

namespace kb {
namespace {

// 32 MiB of scratch, resident on every device that loads the library until the process
// exits.  It holds the three Clenshaw blocks (3 n W floats) and the node marker (n ints).
constexpr size_t FIXED_SCRATCH_BYTES = KB_FIXED_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_fixed_scratch[FIXED_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
constexpr int MAX_M_STEPS = 1024;
std::mutex g_mu;
void *g_scratch_ptr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (set up once per device).
int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= MAX_DEVICES) return fail(KB_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fixed_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(fixed scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return KB_OK;
}

}  // namespace
}  // namespace kb

using namespace kb;

extern "C" int kb_cheb_apply_fixed_scratch(kb_graph *g, kb_phi phi, const kb_params *params,
                                           const int32_t *nodes, int32_t M, int32_t m, float *Y,
                                           void *stream) {
    if (!g || !params || !nodes || !Y) return fail(KB_ERR_ARG, "NULL argument");
    if (M < 1 || M > 128 || M > g->dev.n) return fail(KB_ERR_ARG, "M must be in [1, min(128, n)]");
    if (m < 1 || m > MAX_M_STEPS) return fail(KB_ERR_ARG, "m must be in [1, 1024]");
    if (params->basis != KB_F32) return fail(KB_ERR_UNSUPPORTED, "fixed-scratch solve is FP32 only");
    if (int rc = validate_phi(phi, *params)) return rc;
    for (int i = 0; i < M; ++i) {
        if (nodes[i] < 0 || nodes[i] >= g->dev.n) return fail(KB_ERR_NODES, "node index out of range");
        for (int j = 0; j < i; ++j)
            if (nodes[j] == nodes[i]) return fail(KB_ERR_NODES, "repeated node");
    }
    const int64_t n = g->dev.n;
    const int W = width_for(M);
    const size_t blk = (sizeof(float) * size_t(n) * W + 255) & ~size_t(255);
    const size_t need = 3 * blk + sizeof(int32_t) * size_t(n);
    if (need > FIXED_SCRATCH_BYTES)
        return fail(KB_ERR_ARG, "problem needs " + std::to_string(need) +
                                    " bytes of scratch; the fixed scratch holds " +
                                    std::to_string(FIXED_SCRATCH_BYTES));
    DeviceGuard dg;
    KB_CUDA_TRY(dg.set(g->device));
    void *base = nullptr;
    int rc = scratch_address(g->device, &base);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *bufs[3];
    for (int i = 0; i < 3; ++i) bufs[i] = reinterpret_cast<float *>(static_cast<char *>(base) + i * blk);
    int32_t *marker = reinterpret_cast<int32_t *>(static_cast<char *>(base) + 3 * blk);

    // Lobatto interpolation coefficients of phi on [0, Lambda] (Eq. (chebcoeff)), computed by
    // the routine KB_CHEB uses, into fixed host arrays; the series weights
    // halve c_0 and c_m.
    const double lam = params->lambda_max > 0 ? params->lambda_max : g->lambda;
    double f[MAX_M_STEPS + 1], w[MAX_M_STEPS + 1];
    lobatto_coeffs_into(phi, *params, m, lam, false, f, w);
    w[0] *= 0.5;
    w[m] *= 0.5;

    // Clenshaw: b_m = w_m E_W; b_k = w_k E_W + 2 A b_{k+1} - b_{k+2}; Y = w_0 E_W + A b_1 - b_2,
    // A = I - (2/Lambda) L.  Every buffer that is read is written first in this call.
    KB_CUDA_TRY(cudaMemsetAsync(marker, 0xFF, sizeof(int32_t) * size_t(n), s));
    rc = launch_marker(marker, nodes, M, s);
    if (rc) return rc;
    KB_CUDA_TRY(cudaMemsetAsync(bufs[0], 0, sizeof(float) * size_t(n) * W, s));
    rc = launch_scatter<float>(bufs[0], W, nodes, M, 0, float(w[m]), s);
    if (rc) return rc;
    int cur = 0, prev = -1;
    for (int k = m - 1; k >= 0; --k) {
        const bool last = k == 0;
        int dst = 0;
        while (dst == cur || dst == prev) ++dst;
        LinEpi<float> e;
        e.s1 = (last ? -2.0 : -4.0) / lam;
        e.s0 = last ? 1.0 : 2.0;
        e.s2 = -1.0;
        e.y = prev >= 0 ? bufs[prev] : nullptr;
        e.marker = marker;
        e.wE = w[k];
        if (last) e.yout = Y;
        else e.out = bufs[dst];
        rc = launch_spmm<float>(g->dev, W, bufs[cur], e, s, nullptr, M, prev >= 0 ? 1 : 0,
                                last ? M : 0, last ? M : 0);
        if (rc) return rc;
        prev = cur;
        cur = dst;
    }
    return KB_OK;
}
