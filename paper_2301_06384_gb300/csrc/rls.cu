// RLS kernel predictor from approximated kernel columns (Section 5, Eq.
// (computationcoefficientskrylov); Algorithm 3 for the classical block Lanczos method).
//
//   1. Y ~ phi(L) E_W by one of the five methods (kb_krylov_apply, into scratch);
//   2. the collocation matrix K = E_W^T Y (the rows of Y at the sampling nodes; for cbl this
//      is F_1^T phi(H_m) F_1, the matrix Algorithm 3 solves with, by the proof of
//      Theorem 3.1), and (K + gamma N I) c = y by LU with partial pivoting in FP64 (K is
//      SPD for cbl and cheb2 but may be indefinite or non-symmetric for the other methods,
//      Section 8.3);
//   3. the predictor y_pred = Y c on all n nodes (one streaming pass over Y).
#include <cmath>
#include <vector>

#include "kb_internal.cuh"

namespace kb {
namespace {

constexpr int RLS_THREADS = 256;

// One CTA: gather K, add gamma N on the diagonal, solve by Gaussian elimination with
// partial pivoting (row swaps in shared memory), write c (FP64) and a status.  FP64 is
// slow on this part, so the serial work per column is one pivot search by warp 0 (on the
// order-preserving bit patterns of |a_ik|) and one division; the eliminations and the
// back-substitution updates run on all threads.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return static_cast<unsigned long long>(__double_as_longlong(fabs(v)));
}

__global__ void __launch_bounds__(RLS_THREADS) k_rls_solve(const float *Y, int M,
                                                           const int32_t *nodes,
                                                           const double *labels, double shift,
                                                           double *c, int *status) {
    extern __shared__ double A[];            // [M][M + 1]: K + shift I | y, then rinv[M]
    __shared__ int piv_row, singular;
    __shared__ double inv_piv, xk;
    __shared__ unsigned long long amax_bits;
    const int ld = M + 1;
    double *rinv = A + M * ld;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) { singular = 0; amax_bits = 0ull; }
    __syncthreads();
    unsigned long long my = 0ull;
    for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
        const int i = idx / M, j = idx % M;
        const double v = double(Y[int64_t(nodes[i]) * M + j]) + (i == j ? shift : 0.0);
        A[i * ld + j] = v;
        const unsigned long long bb = abs_bits(v);
        my = bb > my ? bb : my;
    }
    for (int i = threadIdx.x; i < M; i += blockDim.x) A[i * ld + M] = labels[i];
    atomicMax(&amax_bits, my);
    __syncthreads();
    const double tiny = 1e-14 * __longlong_as_double(static_cast<long long>(amax_bits));
    for (int k = 0; k < M; ++k) {
        if (threadIdx.x < 32) {
            unsigned long long best = 0ull;
            int p = k;
            for (int i = k + lane; i < M; i += 32) {
                const unsigned long long bb = abs_bits(A[i * ld + k]);
                if (bb > best) { best = bb; p = i; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int op = __shfl_xor_sync(0xffffffffu, p, off);
                if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
            }
            if (lane == 0) {
                const double a = A[p * ld + k];
                piv_row = p;
                if (!(fabs(a) > tiny)) singular = 1;
                else inv_piv = 1.0 / a;
            }
        }
        __syncthreads();
        if (singular) break;
        const int p = piv_row;
        if (p != k)
            for (int j = threadIdx.x; j <= M; j += blockDim.x) {
                const double t = A[k * ld + j];
                A[k * ld + j] = A[p * ld + j];
                A[p * ld + j] = t;
            }
        __syncthreads();
        const double inv = inv_piv;
        const int rows = M - k - 1, cols = M - k;   // trailing rows, columns k+1..M
        for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
            const int i = k + 1 + idx / cols, j = k + 1 + idx % cols;
            A[i * ld + j] -= (A[i * ld + k] * inv) * A[k * ld + j];
        }
        __syncthreads();
    }
    if (singular) {
        if (threadIdx.x == 0) *status = KB_ERR_BREAKDOWN;
        return;
    }
    // back substitution: reciprocals of the pivots in parallel, then one column sweep per
    // unknown (x_i, then the right-hand sides above it)
    for (int i = threadIdx.x; i < M; i += blockDim.x) rinv[i] = 1.0 / A[i * ld + i];
    __syncthreads();
    for (int i = M - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            xk = A[i * ld + M] * rinv[i];
            A[i * ld + M] = xk;
        }
        __syncthreads();
        const double x = xk;
        for (int j = threadIdx.x; j < i; j += blockDim.x) A[j * ld + M] -= A[j * ld + i] * x;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < M; i += blockDim.x) c[i] = A[i * ld + M];
    if (threadIdx.x == 0) *status = KB_OK;
}

// y_pred[i] = sum_j Y[i, j] c_j; one warp per row group, coefficients split hi + lo float.
__global__ void __launch_bounds__(256) k_rls_predict(const float *Y, int64_t n, int M,
                                                     const double *c, const int *status,
                                                     float *out) {
    if (*status != KB_OK) return;
    __shared__ float ch[128], cl[128];
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        ch[j] = float(c[j]);
        cl[j] = float(c[j] - double(ch[j]));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t row = warp; row < n; row += nwarps) {
        float acc = 0.f;
        for (int j = lane; j < M; j += 32) {
            const float y = Y[row * M + j];
            acc = fmaf(y, ch[j], fmaf(y, cl[j], acc));
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) out[row] = acc;
    }
}

}  // namespace
}  // namespace kb

using namespace kb;

extern "C" int kb_rls_predict(kb_graph *g, kb_method method, kb_phi phi, const kb_params *params,
                              const int32_t *nodes, int32_t M, int32_t m, const double *labels,
                              double gamma, float *y_pred, double *c_host, void *stream,
                              kb_info *info) {
    try {
        if (!g || !params || !nodes || !labels || !y_pred) return fail(KB_ERR_ARG, "NULL argument");
        if (M < 1 || M > 128 || M > g->dev.n) return fail(KB_ERR_ARG, "M must be in [1, min(128, n)]");
        if (!(gamma >= 0) || !std::isfinite(gamma)) return fail(KB_ERR_ARG, "gamma must be >= 0");
        DeviceGuard dg;
        KB_CUDA_TRY(dg.set(g->device));
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int64_t n = g->dev.n;
        // scratch: Y (n x M float), nodes, labels, c, status
        const size_t yb = (sizeof(float) * size_t(n) * M + 255) & ~size_t(255);
        const size_t nb = (sizeof(int32_t) * M + 255) & ~size_t(255);
        const size_t lb = (sizeof(double) * M + 255) & ~size_t(255);
        char *base = nullptr;
        KB_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&base), yb + nb + 2 * lb + 256, s));
        float *Yw = reinterpret_cast<float *>(base);
        int32_t *dn = reinterpret_cast<int32_t *>(base + yb);
        double *dl = reinterpret_cast<double *>(base + yb + nb);
        double *dc = reinterpret_cast<double *>(base + yb + nb + lb);
        int *dst = reinterpret_cast<int *>(base + yb + nb + 2 * lb);
        auto body = [&]() -> int {
            int rc = kb_krylov_apply(g, method, phi, params, nodes, M, m, Yw, stream, info);
            if (rc) return rc;
            KB_CUDA_TRY(cudaMemcpyAsync(dn, nodes, sizeof(int32_t) * M, cudaMemcpyHostToDevice, s));
            KB_CUDA_TRY(cudaMemcpyAsync(dl, labels, sizeof(double) * M, cudaMemcpyHostToDevice, s));
            const size_t smem = sizeof(double) * (size_t(M) * (M + 1) + M);
            static const cudaError_t attr = cudaFuncSetAttribute(
                k_rls_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(double) * (128 * 129 + 128)));
            (void)attr;
            prof_begin(KernelClass::SMALL, s);
            k_rls_solve<<<1, RLS_THREADS, smem, s>>>(Yw, M, dn, dl, gamma * M, dc, dst);
            KB_CUDA_TRY(cudaGetLastError());
            prof_end(KernelClass::SMALL, s, 0, 0);
            const int grid = int(std::min<int64_t>((n + 7) / 8, int64_t(num_sms()) * 8));
            prof_begin(KernelClass::OTHER, s);
            k_rls_predict<<<grid, 256, 0, s>>>(Yw, n, M, dc, dst, y_pred);
            KB_CUDA_TRY(cudaGetLastError());
            prof_end(KernelClass::OTHER, s, double(n) * M * 4 + double(n) * 4, 2.0 * double(n) * M);
            int hst = KB_OK;
            KB_CUDA_TRY(cudaMemcpyAsync(&hst, dst, sizeof(int), cudaMemcpyDeviceToHost, s));
            std::vector<double> hc(static_cast<size_t>(M));
            KB_CUDA_TRY(cudaMemcpyAsync(hc.data(), dc, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
            KB_CUDA_TRY(cudaStreamSynchronize(s));
            if (hst != KB_OK) return fail(hst, "collocation matrix K + gamma N I is singular");
            if (c_host)
                for (int i = 0; i < M; ++i) c_host[i] = hc[i];
            return KB_OK;
        };
        const int rc = body();
        cudaFreeAsync(base, s);
        return rc;
    } catch (const std::bad_alloc &) {
        return fail(KB_ERR_NOMEM, "host allocation failed");
    } catch (...) {
        return fail(KB_ERR_CUDA, "unexpected exception");
    }
}
