// Small dense FP64 kernels and element-wise kernels of the Krylov drivers.
//
//  * k_hkk          symmetrised diagonal block H_kk (Algorithm 1).
//  * k_chol         reduced QR of the new block by CholeskyQR (the reduced QR of Algorithm 1):
//                   Cholesky factor (FP32 first, FP64 fallback), its inverse and the FP64
//                   factor consistent with the applied inverse; the second pass forms H_{k+1,k} = R2 R1
//                   and the transposed block used by the next three-term step (Algorithm 1,
//                   with H_{k-1,k} = H_{k,k-1}^T).  Invariant subspaces stop the process,
//                   rank-deficient blocks report a breakdown (the paper assumes full rank).
//  * k_lanczos_*    scalar recurrences of the global (Algorithm 2) and sequential
//                   (Section 3.3) Lanczos methods: h_kk, h_{k+1,k}, 1/h.
//  * k_tridiag_phi  u = phi(H_m) f_1 for the tridiagonal Lanczos matrices (the projected
//                   step of Algorithm 2; Section 3.3 with phi applied, which its formula omits).
//  * element-wise   unit blocks E_W, node markers, column norms, scaled copies, the
//                   diagonal assembly sum_k u_k Q_k, NaN fill on breakdown.
#include <climits>
#include <type_traits>

#include "kb_internal.cuh"
#include "kb_kernels.cuh"

namespace kb {

// ---------------------------------------------------------------- 16-byte vector access
__device__ __forceinline__ void ldv4(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ldv4(const double *p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void stv4(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void stv4(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void ldv4(const __nv_bfloat16 *p, float (&v)[4]) {
    const uint2 raw = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void stv4(__nv_bfloat16 *p, const float (&v)[4]) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 raw;
    raw.x = *reinterpret_cast<const unsigned int *>(&a);
    raw.y = *reinterpret_cast<const unsigned int *>(&b);
    *reinterpret_cast<uint2 *>(p) = raw;
}
template <typename T> __device__ __forceinline__ double to_double(T v) { return double(v); }
template <> __device__ __forceinline__ double to_double<__nv_bfloat16>(__nv_bfloat16 v) {
    return double(__bfloat162float(v));
}

// ---------------------------------------------------------------- control / init
__global__ void k_ctrl_init(Ctrl *c, int steps) {
    c->status = KB_OK;
    c->stop = 0;
    c->steps = steps;
    c->breakdown_step = -1;
    c->est_change = -1.0;
    c->from_check = -1;
}

template <typename T>
__global__ void k_scatter(T *block, int64_t ld, NodeChunk ch, T val) {
    const int j = threadIdx.x + blockIdx.x * blockDim.x;
    if (j < ch.cnt) block[int64_t(ch.idx[j]) * ld + ch.col0 + j] = val;
}

__global__ void k_marker(int32_t *marker, NodeChunk ch) {
    const int j = threadIdx.x + blockIdx.x * blockDim.x;
    if (j < ch.cnt) marker[ch.idx[j]] = ch.col0 + j;
}

template <typename T>
__global__ void k_scale_copy(T *out, const T *in, int64_t count, double scale) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = T(scale * to_double(in[i]));
}

__global__ void k_fill_nan(float *Y, int64_t n, int64_t ldy, int mo, const Ctrl *ctrl) {
    if (ctrl->status == KB_OK) return;
    const float nanv = __int_as_float(0x7fc00000);
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * mo;
         i += int64_t(gridDim.x) * blockDim.x)
        Y[(i / mo) * ldy + (i % mo)] = nanv;
}

// ---------------------------------------------------------------- cbl small kernels
template <typename T>
__global__ void k_hkk(const double *__restrict__ G, int M, int W, double *__restrict__ Hd,
                      T *__restrict__ C, const Ctrl *ctrl) {
    if (ctrl->stop) return;
    // rows by warp, columns by lane; both loads of an entry issued before any store
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < W; i += nw)
        for (int j = lane; j < W; j += 32) {
            double v = 0.0;
            if (i < M && j < M) v = 0.5 * (__ldg(G + i * W + j) + __ldg(G + j * W + i));
            // recorded exactly as the update subtracts it (rounded to the basis precision)
            const T vt = T(v);
            if (i < M && j < M) Hd[i * M + j] = double(vt);
            C[i * W + j] = vt;
        }
}

// In-place inverse of an upper triangular M x M matrix in shared memory (ld lda), column
// by column: with the leading j x j block already inverted, column j of the inverse is
// -(1/a_jj) X_{0:j,0:j} a_{0:j,j}.  The diagonal reciprocals do not depend on the other
// columns and are formed first, all in parallel; the original entries of column j+1 are
// copied into the second half of t while column j is formed, so each column costs one
// barrier.  Each row's dot product is split over TPR consecutive lanes (TPR = 1, 2, 4 or 8)
// and combined with shuffles.  t: shared scratch of 2 M values.
template <typename S>
__device__ void tri_inv_upper_inplace(S *A, int lda, int M, S *t) {
    int TPR = 1;
    while (TPR < 8 && TPR * 2 * M <= int(blockDim.x)) TPR *= 2;
    const int sub = threadIdx.x % TPR;
    const int row0 = threadIdx.x / TPR;
    const int rstride = blockDim.x / TPR;
    for (int j = threadIdx.x; j < M; j += blockDim.x) A[j * lda + j] = S(1) / A[j * lda + j];
    if (M > 1 && threadIdx.x == 0) t[M] = A[1];   // column 1, row 0
    __syncthreads();
    for (int j = 1; j < M; ++j) {
        const S *tc = (j & 1) ? t + M : t;   // original column j, rows < j
        S *tn = (j & 1) ? t : t + M;         // original column j+1, rows <= j
        if (j + 1 < M)
            for (int i = threadIdx.x; i <= j; i += blockDim.x) tn[i] = A[i * lda + j + 1];
        const S ajj = A[j * lda + j];        // already 1 / a_jj
        // rows i < j, all TPR lanes of a row iterate together (uniform loop bound per warp)
        for (int ib = 0; ib < j; ib += rstride) {
            const int i = ib + row0;
            S acc = S(0);
            if (i < j)
                for (int k = i + sub; k < j; k += TPR) acc = fma(A[i * lda + k], tc[k], acc);
            for (int off = 1; off < TPR; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (i < j && sub == 0) A[i * lda + j] = -ajj * acc;
        }
        __syncthreads();
    }
}

// 1/d for a positive double d by Newton's iteration for the reciprocal, r <- r + r (1 - d r),
// from the single-precision reciprocal: two steps take its 2^-23 relative error to the
// FP64 rounding level (the error squares at each step).  The FP64 division it replaces is
// a long dependent sequence on this part's FP64 unit; this is four FMAs.  Outside the
// normal single-precision range the division is used.
__device__ __forceinline__ double recip_newton(double d) {
    if (!(d > 1e-36 && d < 1e36)) return 1.0 / d;
    double r = double(__frcp_rn(float(d)));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

__device__ __forceinline__ double chol_recip(double d) { return recip_newton(d); }
// the correctly rounded reciprocal (the same value as 1.0f / d, without the division sequence)
__device__ __forceinline__ float chol_recip(float d) { return __frcp_rn(d); }
// 1 / d rounded to nearest in either precision
__device__ __forceinline__ float recip_rn(float d) { return __frcp_rn(d); }
__device__ __forceinline__ double recip_rn(double d) { return 1.0 / d; }

// Scratch of tri_inv_upper_blocked: (P/2)^2 values, P the power of two >= M.
__host__ __device__ inline int tri_inv_tmp_elems(int M) {
    int P = 1;
    while (P < M) P *= 2;
    return (P / 2) * (P / 2);
}

// Blocked in-place inverse of an upper triangular M x M matrix in shared memory (ld lda),
// with few barriers: the 8 x 8 diagonal blocks are inverted one per thread (column by
// column, rows ascending, so each row still reads the original column above the diagonal),
// then pairs of inverted diagonal blocks [A B; 0 C] are merged level by level into
// [A^-1, -A^-1 B C^-1; 0, C^-1] (block edge 8, 16, 32, 64): two barriers per level instead
// of one per column.  tmp: tri_inv_tmp_elems(M) values of shared scratch (the products
// A^-1 B of every pair at the widest level).
template <typename S>
__device__ void tri_inv_upper_blocked(S *A, int lda, int M, S *tmp) {
    const int nb = (M + 7) / 8;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int r0 = b * 8, r1 = min(r0 + 8, M);
        for (int j = r0; j < r1; ++j) {
            const S ajj = recip_rn(A[j * lda + j]);
            for (int i = r0; i < j; ++i) {
                S acc = S(0);
                for (int k = i; k < j; ++k) acc = fma(A[i * lda + k], A[k * lda + j], acc);
                A[i * lda + j] = -ajj * acc;
            }
            A[j * lda + j] = ajj;
        }
    }
    __syncthreads();
    for (int lg = 3, bs = 8; bs < M; ++lg, bs *= 2) {
        // T_p = A_p^-1 B_p for every pair p (rows r0.., columns r0 + bs..); each thread four
        // consecutive columns of one row (four independent FMA chains sharing the A loads)
        const int npairs = (M + 2 * bs - 1) / (2 * bs);
        const int per = bs * bs;
        const int lq = lg - 2;   // log2(bs / 4)
        for (int idx = threadIdx.x; idx < npairs * (per >> 2); idx += blockDim.x) {
            const int p = idx >> (2 * lg - 2), i = (idx >> lq) & (bs - 1), c = (idx & ((bs >> 2) - 1)) << 2;
            const int r0 = p * 2 * bs, cb = min(bs, M - r0 - bs);
            if (cb <= 0 || c >= cb) continue;
            S acc[4] = {S(0), S(0), S(0), S(0)};
            for (int k = i; k < bs; ++k) {
                const S a = A[(r0 + i) * lda + r0 + k];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c + q < cb) acc[q] = fma(a, A[(r0 + k) * lda + r0 + bs + c + q], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) tmp[p * per + i * bs + c + q] = acc[q];
        }
        __syncthreads();
        // B_p <- -T_p C_p^-1 (C^-1 upper triangular: the terms k > c are exact zeros)
        for (int idx = threadIdx.x; idx < npairs * (per >> 2); idx += blockDim.x) {
            const int p = idx >> (2 * lg - 2), i = (idx >> lq) & (bs - 1), c = (idx & ((bs >> 2) - 1)) << 2;
            const int r0 = p * 2 * bs, cb = min(bs, M - r0 - bs);
            if (cb <= 0 || c >= cb) continue;
            const int c0 = r0 + bs;
            S acc[4] = {S(0), S(0), S(0), S(0)};
            const int kend = min(c + 4, cb);
            for (int k = 0; k < kend; ++k) {
                const S t = tmp[p * per + i * bs + k];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c + q < cb) acc[q] = fma(t, A[(c0 + k) * lda + c0 + c + q], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (c + q < cb) A[(r0 + i) * lda + c0 + c + q] = -acc[q];
        }
        __syncthreads();
    }
}

// The upper triangle of an M x M matrix in 4 x 4 tiles: tile t (row-major over the tiles
// (bi, bj), bi <= bj, of the ceil(M/4) x ceil(M/4) grid) -> first row i0, first column j0.
__device__ __forceinline__ void upper_tile(int t, int nt, int &i0, int &j0) {
    int bi = 0;
    while (t >= nt - bi) {
        t -= nt - bi;
        ++bi;
    }
    i0 = 4 * bi;
    j0 = 4 * (bi + t);
}

// C = init + sum_k a(i, k) b(k, j) over the upper triangle i <= j < M of a product of two
// upper triangular M x M matrices, read through the accessors a and b (which must return
// exact zeros below the diagonal).  Each thread takes 4 x 4 tiles of C: 16 independent
// FMA chains over k = i0 .. j0 + 3, the only k where a term of the tile can be non-zero,
// in ascending order, so every entry is the FMA chain of the plain loop k = i .. j with
// exact zero terms added.  epi(i, j, c) receives the upper-triangle entries.
template <typename S, typename FA, typename FB, typename FI, typename FE>
__device__ void tri_mm_upper(int M, const FA &a, const FB &b, const FI &init, const FE &epi) {
    const int nt = (M + 3) / 4;
    const int ntiles = nt * (nt + 1) / 2;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        int i0, j0;
        upper_tile(t, nt, i0, j0);
        S acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                acc[r][q] = (i0 + r < M && j0 + q < M) ? init(i0 + r, j0 + q) : S(0);
        const int kend = min(j0 + 4, M);
        for (int k = i0; k < kend; ++k) {
            S av[4], bv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) av[r] = (i0 + r < M) ? a(i0 + r, k) : S(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) bv[q] = (j0 + q < M) ? b(k, j0 + q) : S(0);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fma(av[r], bv[q], acc[r][q]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + r, j = j0 + q;
                if (i < M && j < M && j >= i) epi(i, j, acc[r][q]);
            }
    }
}

// E = I - S R for upper triangular FP32 matrices S and R in shared memory (ld lda, zeros
// below the diagonal), each entry accumulated as an unevaluated pair of floats: every
// product s r is split exactly into p + pe (p the rounded product, pe = fma(s, r, -p)) and
// subtracted with Knuth's two-sum, so the residual, whose size is the FP32 rounding of the
// inverse, keeps about 48 bits while running on the FP32 pipe.  Returns E rounded to FP32
// through epi(i, j, e) for the upper triangle.
template <typename FE>
__device__ void tri_residual_df(const float *Sm, const float *Rm, int lda, int M, const FE &epi) {
    const int nt = (M + 3) / 4;
    const int ntiles = nt * (nt + 1) / 2;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        int i0, j0;
        upper_tile(t, nt, i0, j0);
        float hi[4][4], lo[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                hi[r][q] = (i0 + r == j0 + q) ? 1.f : 0.f;
                lo[r][q] = 0.f;
            }
        const int kend = min(j0 + 4, M);
        for (int k = i0; k < kend; ++k) {
            float sv[4], rv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) sv[r] = (i0 + r < M) ? Sm[(i0 + r) * lda + k] : 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) rv[q] = (j0 + q < M) ? Rm[k * lda + j0 + q] : 0.f;
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float p = __fmul_rn(sv[r], rv[q]);
                    const float pe = fmaf(sv[r], rv[q], -p);
                    float s, e;
                    two_sum(hi[r][q], -p, s, e);
                    hi[r][q] = s;
                    lo[r][q] += e - pe;
                }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + r, j = j0 + q;
                if (i < M && j < M && j >= i) epi(i, j, hi[r][q] + lo[r][q]);
            }
    }
}

// Copy an M x M row-major matrix (leading dimension ldg) from global memory through
// store(i, j, v): rows by warp, columns by lane (coalesced), eight rows in flight per warp
// before their stores.
template <typename FS>
__device__ __forceinline__ void load_square(const double *g, int ldg, int M, const FS &store) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i0 = warp; i0 < M; i0 += 8 * nw)
        for (int j = lane; j < M; j += 32) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * nw;
                v[u] = i < M ? __ldg(g + i * ldg + j) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * nw;
                if (i < M) store(i, j, v[u]);
            }
        }
}

// Cholesky G = R^T R of an M x M symmetric matrix in shared memory, upper R overwriting A
// and the lower part zeroed.  Square-root-free form: step j needs the pivot d_j (the
// diagonal of the current Schur complement) and one reciprocal; the Schur complement update
// is A_ab -= u_ja u_jb / d_j with the unscaled pivot row u_j.  The square roots and the row
// scaling R_j = u_j / sqrt(d_j) are applied at the end, for all rows at once.  Look-ahead:
// during step j warp 0 updates only the next pivot row j+1, takes its pivot and the one
// FP64 division and forms the scaled row u_{j+1} / d_{j+1} (into the other half of a double
// buffer), while the other warps update rows j+2..; so each column costs one barrier and
// the division overlaps the bulk of the update.  Returns false (all threads) on a pivot
// <= piv_rel2 * max diag.  t: shared scratch of 3 M doubles.  Needs blockDim.x >= 64.
// bad: two shared flags, zero on entry.  The failure of pivot j is recorded in bad[j & 1]
// (by warp 0 during step j-1) and read by every thread at the top of step j, after the
// barrier that ends step j-1; the flag warp 0 writes during step j is the other one, so no
// thread can read a flag in the same barrier interval in which it is written (all threads
// leave at the same step).
template <typename S>
__device__ bool chol_upper_inplace(S *A, int lda, int M, S piv_rel2, S maxdiag, S *t, int *bad) {
    S *const srow0 = t, *const srow1 = t + M;   // u_j / d_j, double-buffered by the parity of j
    S *piv = t + 2 * M;        // d_j
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const S thr = piv_rel2 * maxdiag;
    // pivot row 0
    if (warp == 0) {
        const S d = A[0];
        if (!(d > thr)) {
            if (lane == 0) bad[0] = 1;
        } else {
            const S dinv = chol_recip(d);
            for (int c = 1 + lane; c < M; c += 32) srow0[c] = A[c] * dinv;
            if (lane == 0) piv[0] = d;
        }
    }
    __syncthreads();
    for (int j = 0; j < M; ++j) {
        if (bad[j & 1]) return false;
        const S *sr = (j & 1) ? srow1 : srow0;
        if (warp == 0) {
            if (j + 1 < M) {
                // the next pivot row: A[j+1][c] -= u_{j,j+1} u_{j,c} / d_j, c >= j+1, held in
                // registers (lane l: c = j+1+l+32q); its pivot comes from lane 0 by a shuffle
                const S ujn = A[j * lda + j + 1];
                S v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = j + 1 + lane + 32 * q;
                    v[q] = c < M ? fma(-ujn, sr[c], A[(j + 1) * lda + c]) : S(0);
                }
                const S d = __shfl_sync(0xffffffffu, v[0], 0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = j + 1 + lane + 32 * q;
                    if (c < M) A[(j + 1) * lda + c] = v[q];
                }
                if (!(d > thr)) {
                    if (lane == 0) bad[(j + 1) & 1] = 1;
                } else {
                    const S dinv = chol_recip(d);
                    S *sn = ((j + 1) & 1) ? srow1 : srow0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c = j + 1 + lane + 32 * q;
                        if (c >= j + 2 && c < M) sn[c] = v[q] * dinv;
                    }
                    if (lane == 0) piv[j + 1] = d;
                }
            }
        } else {
            // rows j+2.. of the trailing upper triangle: rows by warp, columns by lane (c =
            // lane + 32q); four rows' loads are issued before any of their stores
            const int nw = (blockDim.x >> 5) - 1;
            S srv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) srv[q] = lane + 32 * q < M ? sr[lane + 32 * q] : S(0);
            for (int ra0 = j + 1 + warp; ra0 < M; ra0 += 4 * nw) {
                S u[4], a[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int ra = ra0 + r * nw;
                    u[r] = ra < M ? A[j * lda + ra] : S(0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c = lane + 32 * q;
                        a[r][q] = (ra < M && c >= ra && c < M) ? A[ra * lda + c] : S(0);
                    }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int ra = ra0 + r * nw;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c = lane + 32 * q;
                        if (ra < M && c >= ra && c < M) A[ra * lda + c] = fma(-u[r], srv[q], a[r][q]);
                    }
                }
            }
        }
        __syncthreads();
    }
    // (no pivot is examined during the last step: the flags are final here)
    if (bad[0] | bad[1]) return false;
    // R_jj = sqrt(d_j), R_jc = u_jc / sqrt(d_j)
    S *rinv = srow0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const S r = sqrt(piv[j]);
        piv[j] = r;
        rinv[j] = recip_rn(r);
    }
    __syncthreads();
    for (int i = warp; i < M; i += blockDim.x >> 5)
        for (int j = lane; j < M; j += 32) {
            if (j < i) A[i * lda + j] = S(0);
            else if (j == i) A[i * lda + j] = piv[i];
            else A[i * lda + j] *= rinv[i];
        }
    __syncthreads();
    return true;
}

// Reduced QR of the new block by CholeskyQR (Algorithm 1), pass 1 or 2 of
// CholeskyQR2.  Outputs: Rinv (W x W, basis precision) applied by the row-block kernels;
// pass 1 records R1 = the FP64 inverse of the applied inverse; pass 2 records
// H_{k+1,k} = R2 R1 (rounded to the basis precision) and B = H^T.
//
// Pass 1 (G = X^T X, any conditioning): FP64 Cholesky; in the FP32 path the inverse is
// formed in FP32 from R1 and R1 is then recomputed as the FP64 inverse of that FP32
// inverse, so that X = X1 R1 holds for the applied matrices.
// Pass 2 of the FP32 path (G = I + E, ||E|| of the order of the FP32 rounding of pass 1):
// to first order R2 = I + Phi(E) with Phi = strict upper part plus half the diagonal,
// R2^{-1} = I - Phi(E) (the orthogonality of Q = X1 (I - Phi(E)) is then I + O(||E||^2));
// the applied inverse I - F has the inverse I + F + F^2 + O(F^3), so H = R1 + F R1 + F (F R1),
// the corrections formed in FP32.  When ||E|| is not small (max |E_ij| >= 1e-4), and always
// in the FP64 mode, pass 2 uses the pass-1 algorithm.
//
// The kernel runs on one SM, so its time is latency: the matrices are loaded with several
// loads in flight per thread, the triangular products run as 4 x 4 register tiles (16
// independent FMA chains per thread instead of one serial chain per entry), the residual of
// the FP32 inverse uses pairs of floats rather than FP64 (whose rate on this part is a small
// fraction of FP32), the statistics of G are reduced in parallel (max |E_ij| through the
// order-preserving bit patterns of non-negative doubles) and the Cholesky factorisation needs
// one division per column.
constexpr int CHOL_NEWTON_MAX = 64;   // widest block with the corrected-inverse scratch
template <typename T>
__global__ void __launch_bounds__(256) k_chol(const double *G, int M, int W, int pass, int step,
                                              double inv_thresh2, double piv_rel2, double *R1,
                                              T *Rinv, double *Hs, T *Bout, Ctrl *ctrl) {
    if (ctrl->stop) return;
    // [M][M+1] FP64, then [M][M+1] T, then 3 M + 2 doubles of scratch
    extern __shared__ __align__(16) double A[];
    __shared__ int bad, small;
    __shared__ int pivot_bad[2];   // chol_upper_inplace's per-parity pivot failure flags
    __shared__ double maxdiag;
    __shared__ unsigned long long emax_bits;
    const int lda = M + 1;
    T *Sf = reinterpret_cast<T *>(A + M * lda);
    double *t = reinterpret_cast<double *>(Sf + M * lda + (sizeof(T) == 4 ? (M * lda) % 2 : 0));
    const bool try_small = pass == 2 && sizeof(T) == 4;
    if (threadIdx.x == 0) {
        emax_bits = 0ull;
        bad = 0;
        pivot_bad[0] = 0;
        pivot_bad[1] = 0;
    }
    __syncthreads();
    unsigned long long my_e = 0ull;
    load_square(G, W, M, [&](int i, int j, double g) {
        A[i * lda + j] = g;
        if (try_small) {
            double e = g;
            if (i == j) e -= 1.0;
            const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(fabs(e)));
            my_e = b > my_e ? b : my_e;
        }
    });
    if (try_small) {
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, my_e, off);
            my_e = o > my_e ? o : my_e;
        }
        if ((threadIdx.x & 31) == 0) atomicMax(&emax_bits, my_e);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // trace and largest diagonal entry (non-negative for a Gram matrix: bit order)
        double tr = 0.0;
        unsigned long long mx = 0ull;
        for (int i = threadIdx.x; i < M; i += 32) {
            const double d = A[i * lda + i];
            tr += d;
            const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(fabs(d)));
            mx = b > mx ? b : mx;
        }
        for (int off = 16; off > 0; off >>= 1) {
            tr += __shfl_xor_sync(0xffffffffu, tr, off);
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
            mx = o > mx ? o : mx;
        }
        if (threadIdx.x == 0) {
            maxdiag = __longlong_as_double(static_cast<long long>(mx));
            small = (try_small && __longlong_as_double(static_cast<long long>(emax_bits)) < 1e-4) ? 1 : 0;
            if (pass == 1 && !(tr > inv_thresh2)) {
                // X vanished: the block Krylov space is invariant; keep the blocks so far
                ctrl->stop = 1;
                ctrl->steps = step;
                bad = 2;
            }
        }
    }
    __syncthreads();
    if (bad) return;
    if (small) {
        // ---- pass 2, first order (FP32 path): S = I - Phi(E) applied; F = I - S exactly
        for (int i = threadIdx.x >> 5; i < W; i += blockDim.x >> 5)
            for (int j = threadIdx.x & 31; j < W; j += 32) {
                const int idx = i * W + j;
                // one FP64 subtraction per entry (E is small: the rest is exact or FP32-level)
                T v = T(0);
                if (i < M && j < M && j >= i) {
                    const float e = float(A[i * lda + j] - (i == j ? 1.0 : 0.0));
                    v = (i == j) ? T(1.f - 0.5f * e) : T(-e);
                }
                Rinv[idx] = v;
                if (i < M && j < M) Sf[i * lda + j] = (j >= i) ? T((i == j ? 1.f : 0.f) - float(v)) : T(0);
            }
        __syncthreads();
        // A is free now: R1 rounded to T, and C = F R1 (both upper triangular, zeros below)
        T *R1t = reinterpret_cast<T *>(A);
        T *Ct = R1t + M * lda;
        load_square(R1, M, M, [&](int i, int j, double v) {
            R1t[i * lda + j] = (j >= i) ? T(v) : T(0);
            Ct[i * lda + j] = T(0);
        });
        __syncthreads();
        auto sf = [&](int i, int k) { return Sf[i * lda + k]; };
        auto zero = [](int, int) { return T(0); };
        tri_mm_upper<T>(M, sf, [&](int k, int j) { return R1t[k * lda + j]; }, zero,
                        [&](int i, int j, T c) { Ct[i * lda + j] = c; });
        // entries of Hs and B outside H's upper triangle are zero
        for (int i = threadIdx.x >> 5; i < W; i += blockDim.x >> 5)
            for (int j = threadIdx.x & 31; j < W; j += 32) {
                if (i < M && j < M && j >= i) continue;
                if (i < M && j < M) Hs[i * M + j] = 0.0;
                Bout[j * W + i] = T(0);
            }
        __syncthreads();
        // H = (I + F + F^2) R1 = R1 + (C + F C), the corrections of relative size ||E||
        tri_mm_upper<T>(M, sf, [&](int k, int j) { return Ct[k * lda + j]; }, zero,
                        [&](int i, int j, T corr2) {
                            const double h = __ldg(R1 + i * M + j) + double(Ct[i * lda + j] + corr2);
                            const T ht = T(h);
                            Hs[i * M + j] = double(ht);
                            Bout[j * W + i] = ht;
                        });
        return;
    }
    // ---- general CholeskyQR pass
    // Pass 1 of the FP32 path first factors G in FP32 (the FP32 pipe runs 64 times the FP64
    // rate): the first pass only has to bring X close to orthonormal, the second pass
    // corrects what is left (its first-order form when max |G2 - I| < 1e-4, a full
    // factorisation otherwise), and R1 below is the FP64 inverse of the applied inverse
    // whatever R it came from.  A pivot below 1e-5 of the largest diagonal entry is not
    // trusted in FP32: the factorisation is then redone in FP64 (which alone decides a
    // breakdown).
    bool factored = false;
    if (sizeof(T) == 4 && pass == 1) {
        float *Af = reinterpret_cast<float *>(Sf);   // Sf is free until the inverse below
        float *tf = reinterpret_cast<float *>(t);
        for (int i = threadIdx.x >> 5; i < M; i += blockDim.x >> 5)
            for (int j = threadIdx.x & 31; j < M; j += 32) {
                Af[i * lda + j] = float(A[i * lda + j]);
            }
        __syncthreads();
        if (chol_upper_inplace<float>(Af, lda, M, 1e-5f, float(maxdiag), tf, pivot_bad)) {
            for (int i = threadIdx.x >> 5; i < M; i += blockDim.x >> 5)
                for (int j = threadIdx.x & 31; j < M; j += 32) {
                    A[i * lda + j] = (j >= i) ? double(Af[i * lda + j]) : 0.0;
                }
            factored = true;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            pivot_bad[0] = 0;
            pivot_bad[1] = 0;
        }
        __syncthreads();
    }
    if (!factored && !chol_upper_inplace<double>(A, lda, M, piv_rel2, maxdiag, t, pivot_bad)) {
        if (threadIdx.x == 0) {
            ctrl->status = KB_ERR_BREAKDOWN;
            ctrl->stop = 1;
            ctrl->steps = step;
            ctrl->breakdown_step = step;
        }
        return;
    }
    const bool newton = sizeof(T) == 4 && M <= CHOL_NEWTON_MAX;
    double *Sd = t + 3 * M + 2;                               // [M][M+1] (newton only)
    float *Rf = reinterpret_cast<float *>(Sd + M * lda);      // [M][M+1]
    float *C1 = Rf + M * lda;                                 // [M][M+1]
    for (int i = threadIdx.x >> 5; i < M; i += blockDim.x >> 5)
        for (int j = threadIdx.x & 31; j < M; j += 32) {
            Sf[i * lda + j] = T(A[i * lda + j]);
            if (newton) Rf[i * lda + j] = float(Sf[i * lda + j]);
        }
    __syncthreads();
    {
        // scratch after the Newton region (launch_chol sizes it)
        unsigned char *after = reinterpret_cast<unsigned char *>(t + 3 * M + 2) + (newton ? 16 * size_t(M) * lda : 0);
        tri_inv_upper_blocked<T>(Sf, lda, M, reinterpret_cast<T *>(after));
    }
    for (int i = threadIdx.x >> 5; i < W; i += blockDim.x >> 5)
        for (int j = threadIdx.x & 31; j < W; j += 32) {
            const int idx = i * W + j;
            Rinv[idx] = (i < M && j < M && j >= i) ? Sf[i * lda + j] : T(0);
        }
    if (sizeof(T) == 4) {
        // R := the FP64 inverse of the applied FP32 inverse S.
        bool exact = !newton;
        if (newton) {
            // With S R = I - E (E upper triangular, of the order of the FP32 rounding),
            // S^{-1} = R (I - E)^{-1} = R + R E + R E^2 + O(E^3): E is formed from S and R with
            // a residual more precise than FP32 (pairs of floats when R is the FP32 factor,
            // FP64 when the factorisation fell back to FP64), the corrections in FP32.  When
            // max |E_ij| >= 1e-3 the exact FP64 inverse below is used instead.
            __shared__ unsigned int emax_e;
            float *Sff = reinterpret_cast<float *>(Sf);
            // E goes to the Sd region (pair residual; S stays in Sf) or, with the FP64
            // residual, which reads S from Sd, over S in Sf
            float *Ef = factored ? reinterpret_cast<float *>(Sd) : Sff;
            if (threadIdx.x == 0) emax_e = 0u;
            for (int i = threadIdx.x >> 5; i < M; i += blockDim.x >> 5)
                for (int j = threadIdx.x & 31; j < M; j += 32) {
                    if (factored) {
                        if (j < i) Ef[i * lda + j] = 0.f;
                    } else {
                        Sd[i * lda + j] = (j >= i) ? double(Sff[i * lda + j]) : 0.0;
                    }
                }
            __syncthreads();
            unsigned int my = 0u;
            auto put_e = [&](int i, int j, float ef) {
                Ef[i * lda + j] = ef;
                const unsigned int bits = __float_as_uint(fabsf(ef));
                my = bits > my ? bits : my;
            };
            if (factored) {
                tri_residual_df(Sff, Rf, lda, M, put_e);
            } else {
                tri_mm_upper<double>(
                    M, [&](int i, int k) { return -Sd[i * lda + k]; }, [&](int k, int j) { return A[k * lda + j]; },
                    [](int i, int j) { return i == j ? 1.0 : 0.0; },
                    [&](int i, int j, double e) { put_e(i, j, float(e)); });
            }
            atomicMax(&emax_e, my);
            __syncthreads();
            if (__uint_as_float(emax_e) < 1e-3f) {
                auto ef = [&](int k, int j) { return Ef[k * lda + j]; };
                auto zero = [](int, int) { return 0.f; };
                for (int i = threadIdx.x >> 5; i < M; i += blockDim.x >> 5)
                    for (int j = threadIdx.x & 31; j < M; j += 32) {
                        if (j < i) C1[i * lda + j] = 0.f;
                    }
                tri_mm_upper<float>(M, [&](int i, int k) { return Rf[i * lda + k]; }, ef, zero,
                                    [&](int i, int j, float c) { C1[i * lda + j] = c; });
                __syncthreads();
                tri_mm_upper<float>(M, [&](int i, int k) { return C1[i * lda + k]; }, ef, zero,
                                    [&](int i, int j, float c2) { A[i * lda + j] += double(C1[i * lda + j] + c2); });
                __syncthreads();
            } else {
                exact = true;
                for (int i = threadIdx.x >> 5; i < M; i += blockDim.x >> 5)
                    for (int j = threadIdx.x & 31; j < M; j += 32) {
                        A[i * lda + j] = factored ? ((j >= i) ? double(Sff[i * lda + j]) : 0.0) : Sd[i * lda + j];
                    }
                __syncthreads();
            }
        } else {
            for (int i = threadIdx.x >> 5; i < M; i += blockDim.x >> 5)
                for (int j = threadIdx.x & 31; j < M; j += 32) {
                    A[i * lda + j] = (j >= i) ? double(Sf[i * lda + j]) : 0.0;
                }
            __syncthreads();
        }
        if (exact) tri_inv_upper_inplace<double>(A, lda, M, t);
    }
    // (FP64 basis: the inverse is applied in FP64, R needs no correction)
    if (pass == 1) {
        for (int i = threadIdx.x >> 5; i < M; i += blockDim.x >> 5)
            for (int j = threadIdx.x & 31; j < M; j += 32) {
                const int idx = i * M + j;
                R1[idx] = (j >= i) ? A[i * lda + j] : 0.0;
            }
    } else {
        // H_{k+1,k} = R2 R1 (upper triangular); B = H^T for the next three-term step.  H is
        // recorded rounded to the basis precision, i.e. exactly as the next step subtracts it.
        for (int i = threadIdx.x >> 5; i < W; i += blockDim.x >> 5)
            for (int j = threadIdx.x & 31; j < W; j += 32) {
                if (i < M && j < M && j >= i) continue;
                if (i < M && j < M) Hs[i * M + j] = 0.0;
                Bout[j * W + i] = T(0);
            }
        tri_mm_upper<double>(
            M, [&](int i, int k) { return A[i * lda + k]; }, [&](int k, int j) { return __ldg(R1 + k * M + j); },
            [](int, int) { return 0.0; },
            [&](int i, int j, double h) {
                const T ht = T(h);
                Hs[i * M + j] = double(ht);
                Bout[j * W + i] = ht;
            });
    }
}

// ---------------------------------------------------------------- full reorthogonalisation
// "Twice is enough" (Kahan's criterion, as given in Parlett's The Symmetric Eigenvalue
// Problem): after one classical Gram-Schmidt pass x_1 = x_0 - Q Q^T x_0, x_1 is orthogonal to
// Q to working precision when ||x_1|| >= ||x_0|| / sqrt(2); otherwise a second pass is
// needed.  Applied column by column to the block: the squared column norms of X before the
// first pass (the diagonal of its Gram) are saved, and after the pass the second one is
// skipped (*skip = 1) when every column kept at least half of its squared norm.
__global__ void k_reorth_save(const double *G, int M, int W, double *d0) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) d0[i] = G[int64_t(i) * W + i];
}
__global__ void k_reorth_decide(const double *G, const double *d0, int M, int W, int32_t *skip) {
    bool ok = true;
    for (int i = threadIdx.x; i < M; i += 32) ok = ok && G[int64_t(i) * W + i] >= 0.5 * d0[i];
    ok = __all_sync(0xffffffffu, ok);
    if (threadIdx.x == 0) *skip = ok ? 1 : 0;
}

int launch_reorth_save(const double *G, int M, int W, double *d0, cudaStream_t s) {
    k_reorth_save<<<1, 128, 0, s>>>(G, M, W, d0);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}
int launch_reorth_decide(const double *G, const double *d0, int M, int W, int32_t *skip, cudaStream_t s) {
    k_reorth_decide<<<1, 32, 0, s>>>(G, d0, M, W, skip);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

// ---------------------------------------------------------------- gbl / sbl scalars
// Reduce [nparts][W] partials per column (fixed order) into s[W].  df: the partials are
// double-float pairs (FP32 arithmetic), combined on the FP32 pipe; else doubles.
__device__ void reduce_cols(const double *parts, int nparts, int W, double *s, int df) {
    // one warp per strided subset of the partials (up to 32 warps), eight loads in flight per
    // lane (each into its own accumulator, merged in a fixed order), then a fixed-order
    // combination of the warps' sums
    __shared__ double tmp[32][128];
    constexpr int U = 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < W; c0 += 32) {
        const int c = c0 + lane;
        if (c >= W) continue;
        if (df) {
            const DF *pp = reinterpret_cast<const DF *>(parts);
            DF a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) a[u] = DF{0.f, 0.f};
            int p = warp;
            for (; p < nparts; p += U * nw) {
                DF v[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    v[u] = p + u * nw < nparts ? pp[int64_t(p + u * nw) * W + c] : DF{0.f, 0.f};
#pragma unroll
                for (int u = 0; u < U; ++u) df_merge(a[u], v[u]);
            }
#pragma unroll
            for (int u = 1; u < U; ++u) df_merge(a[0], a[u]);
            reinterpret_cast<DF *>(&tmp[warp][0])[c] = a[0];
        } else {
            double a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) a[u] = 0.0;
            int p = warp;
            for (; p < nparts; p += U * nw) {
                double v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = p + u * nw < nparts ? parts[int64_t(p + u * nw) * W + c] : 0.0;
#pragma unroll
                for (int u = 0; u < U; ++u) a[u] += v[u];
            }
            double t = a[0];
#pragma unroll
            for (int u = 1; u < U; ++u) t += a[u];
            tmp[warp][c] = t;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        if (df) {
            DF t = reinterpret_cast<const DF *>(&tmp[0][0])[c];
            for (int w = 1; w < nw; ++w) df_merge(t, reinterpret_cast<const DF *>(&tmp[w][0])[c]);
            s[c] = df_value(t);
        } else {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += tmp[w][c];
            s[c] = t;
        }
    }
    __syncthreads();
}

// Scale factors sigma (Q_k = sigma_k P_k) are rounded to the basis precision when the
// basis is FP32, so that the SpMM applies exactly the sigma the recurrence records.
__device__ __forceinline__ double round_to(double v, int round32) {
    return round32 ? double(float(v)) : v;
}

__global__ void k_lanczos_init(int W, int M, int gbl, int round32, double *sigma, int32_t *alive,
                               double *c1, double *c2) {
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        const bool live = c < M;
        const double s0 = live ? round_to(gbl ? 1.0 / sqrt(double(M)) : 1.0, round32) : 0.0;
        sigma[c] = s0;
        alive[c] = live ? 1 : 0;
        c1[c] = s0;
        c2[c] = 0.0;
    }
}

// Sum of s[0..M) by warp 0 (fixed order); the result is returned to lane 0.
__device__ __forceinline__ double warp0_sum(const double *s, int M) {
    double t = 0.0;
    for (int c = threadIdx.x; c < M; c += 32) t += s[c];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    return t;
}

// alpha_k = <Q_k, X> (gbl: Frobenius, sbl: per column) from SpMM dot partials of P_k . X
__global__ void k_lanczos_alpha(const double *parts, int nparts, int W, int M, int gbl, int k,
                                int df, const double *sigma, double *alpha, double *a_upd,
                                const Ctrl *ctrl) {
    if (ctrl->stop) return;
    __shared__ double s[128];
    reduce_cols(parts, nparts, W, s, df);
    const double *sg = sigma + int64_t(k) * W;
    if (gbl) {
        __shared__ double tot;
        if (threadIdx.x < 32) {
            const double t = warp0_sum(s, M);
            if (threadIdx.x == 0) tot = sg[0] * t;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            alpha[int64_t(k) * W + c] = c < M ? tot : 0.0;
            a_upd[c] = c < M ? tot * sg[0] : 0.0;
        }
    } else {
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            const double al = c < M ? sg[c] * s[c] : 0.0;
            alpha[int64_t(k) * W + c] = al;
            a_upd[c] = al * sg[c];
        }
    }
}

// beta_{k+1} = ||X|| (gbl: Frobenius, sbl: per column), sigma_{k+1} = 1/beta, and the
// SpMM coefficients of the next step: X = sigma_{k+1} L P_{k+1} - beta_{k+1} sigma_k P_k.
// sigma_{k+1} is rounded to the basis precision and beta_{k+1} is recorded as its exact
// reciprocal, so Q_{k+1} = sigma_{k+1} P_{k+1} = X / beta_{k+1} holds for the stored values.
__global__ void k_lanczos_beta(const double *parts, int nparts, int W, int M, int gbl, int k,
                               int round32, double thresh, double *beta, double *sigma,
                               int32_t *alive, double *c1, double *c2, Ctrl *ctrl) {
    if (ctrl->stop) return;
    __shared__ double s[128];
    reduce_cols(parts, nparts, W, s, round32);
    const double *sk = sigma + int64_t(k) * W;
    double *sn = sigma + int64_t(k + 1) * W;
    double *bn = beta + int64_t(k + 1) * W;
    if (gbl) {
        __shared__ double b;
        __shared__ int stop;
        if (threadIdx.x < 32) {
            const double t = warp0_sum(s, M);
            if (threadIdx.x == 0) {
                b = sqrt(t);
                stop = !(b > thresh);
                if (stop) { ctrl->stop = 1; ctrl->steps = k + 1; }
            }
        }
        __syncthreads();
        const double sg = round_to(1.0 / b, round32);
        const double bt = 1.0 / sg;
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            const bool live = c < M && !stop;
            bn[c] = live ? bt : 0.0;
            sn[c] = live ? sg : 0.0;
            c1[c] = live ? sg : 0.0;
            c2[c] = live ? -bt * sk[c] : 0.0;
        }
    } else {
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            const double b = sqrt(s[c]);
            const bool live = c < M && alive[c] && (b > thresh);
            if (!live) alive[c] = 0;
            const double sg = live ? round_to(1.0 / b, round32) : 0.0;
            const double bt = live ? 1.0 / sg : 0.0;
            bn[c] = bt;
            sn[c] = sg;
            c1[c] = sg;
            c2[c] = live ? -bt * sk[c] : 0.0;
        }
    }
}

// u = phi(T) e_1 for each column's tridiagonal T (diag alpha_k, off-diagonal beta_{k+1}),
// then assembly weights omega_k[c] = scale * u_k * sigma_k[c].
//   exp:    Chebyshev series of e^{-t lambda} on [0, Lambda] in T_j(I - 2T/Lambda)
//   spline: s_int solves with the SPD tridiagonal eps I + T (Thomas algorithm; the
//           factorisation is formed once and reused by the s_int solves)
// One CTA per tridiagonal (column c; a single one for the global method), its threads
// parallel over the rows of the three-term recurrence.  The vectors live in shared memory
// when 6 m doubles fit (m <= TRI_SMEM_M), else in the global scratch work (4 m per column).
constexpr int TRI_SMEM_M = 1024;
constexpr int TRI_THREADS = 128;

// Chebyshev series of e^{-t lambda} applied to e_1, terms [j0, j0 + cc.n) of it, for series
// longer than one ChebCoef: V_j (term j) lives in slot j % 3 of the column's global state
// (3 m doubles), the partial sum u in the fourth m doubles (the layout k_tridiag_phi reads
// with u_ready).  A = I - (2/lam) T; V_0 = e_1, V_1 = A e_1, V_j = 2 A V_{j-1} - V_{j-2}.
__global__ void __launch_bounds__(TRI_THREADS) k_tridiag_exp_chunk(int W, int M, int m, int gbl,
                                                                   const double *alpha,
                                                                   const double *beta, double lam,
                                                                   ChebCoef cc, int j0,
                                                                   double *work, const Ctrl *ctrl) {
    const int c = blockIdx.x;
    if (c >= (gbl ? 1 : M)) return;
    const int s = gbl ? ctrl->steps : m;
    double *slot[3] = {work + int64_t(c) * 4 * m, work + int64_t(c) * 4 * m + m, work + int64_t(c) * 4 * m + 2 * m};
    double *u = work + int64_t(c) * 4 * m + 3 * m;
    auto a_of = [&](int k) { return alpha[int64_t(k) * W + c]; };
    auto b_of = [&](int k) { return beta[int64_t(k) * W + c]; };
    const double g = 2.0 / lam;
    for (int q = 0; q < cc.n; ++q) {
        const int j = j0 + q;
        double *vn = slot[j % 3];
        if (j == 0) {
            for (int k = threadIdx.x; k < m; k += blockDim.x) {
                vn[k] = k == 0 ? 1.0 : 0.0;
                u[k] = k == 0 ? cc.d[q] : 0.0;
                slot[1][k] = 0.0;
                slot[2][k] = 0.0;
            }
        } else {
            const double *pc = slot[(j - 1) % 3];
            const double *pp = slot[(j + 1) % 3];   // V_{j-2} (slot (j - 2) % 3)
            for (int k = threadIdx.x; k < s; k += blockDim.x) {
                double tv = a_of(k) * pc[k];
                if (k > 0) tv += b_of(k) * pc[k - 1];
                if (k + 1 < s) tv += b_of(k + 1) * pc[k + 1];
                const double av = pc[k] - g * tv;
                const double v = j == 1 ? av : 2.0 * av - pp[k];
                vn[k] = v;
                u[k] += cc.d[q] * v;
            }
        }
        __syncthreads();
    }
}

// u_ready: the series part of e^{-t T} e_1 was formed by k_tridiag_exp_chunk in work; only
// the bound check and the scaling into omega run here.
__global__ void __launch_bounds__(TRI_THREADS) k_tridiag_phi(int W, int M, int m, int gbl,
                                                             const double *alpha,
                                                             const double *beta,
                                                             const double *sigma, int phi_kind,
                                                             double eps, int s_int, double lam,
                                                             TriCoef tc, double *omega,
                                                             double *work, double *qwork,
                                                             Ctrl *ctrl, double bound, int u_ready) {
    const ChebCoef &cc = tc.cc;
    const int c = blockIdx.x;
    const int ncol = gbl ? 1 : M;
    if (c >= ncol) {
        for (int k = threadIdx.x; k < m; k += blockDim.x) omega[int64_t(k) * W + c] = 0.0;
        return;
    }
    const int s = gbl ? ctrl->steps : m;
    extern __shared__ __align__(16) double tsm[];
    const bool in_smem = m <= TRI_SMEM_M && !u_ready;
    double *v0, *v1, *v2, *u;
    const double *av, *bv;
    int64_t st;   // stride of av / bv
    if (in_smem) {
        v0 = tsm; v1 = v0 + m; v2 = v1 + m; u = v2 + m;
        double *a_s = u + m, *b_s = a_s + m;
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            a_s[k] = alpha[int64_t(k) * W + c];
            b_s[k] = beta[int64_t(k) * W + c];
        }
        av = a_s; bv = b_s; st = 1;
    } else {
        v0 = work + int64_t(c) * 4 * m; v1 = v0 + m; v2 = v1 + m; u = v2 + m;
        av = alpha + c; bv = beta + c; st = W;
    }
    // b_of(k) couples rows k-1 and k
    auto a_of = [&](int k) { return av[int64_t(k) * st]; };
    auto b_of = [&](int k) { return bv[int64_t(k) * st]; };
    if (!u_ready)
        for (int k = threadIdx.x; k < m; k += blockDim.x) { v0[k] = 0.0; v1[k] = 0.0; v2[k] = 0.0; u[k] = 0.0; }
    __syncthreads();
    if (u_ready) {
        // (series formed in chunks)
    } else if (phi_kind == KB_PHI_EXP) {
        // v0 = e_1, v1 = A e_1, v_{j+1} = 2 A v_j - v_{j-1}, A = I - (2/lam) T
        const double g = 2.0 / lam;
        if (threadIdx.x == 0) { v0[0] = 1.0; u[0] = cc.d[0]; }
        __syncthreads();
        double *pp = v0, *pc = v1, *pn = v2;
        for (int k = threadIdx.x; k < s; k += blockDim.x) {
            double tv = a_of(k) * pp[k];
            if (k > 0) tv += b_of(k) * pp[k - 1];
            if (k + 1 < s) tv += b_of(k + 1) * pp[k + 1];
            pc[k] = pp[k] - g * tv;
            u[k] += cc.d[1] * pc[k];
        }
        __syncthreads();
        for (int j = 2; j < cc.n; ++j) {
            for (int k = threadIdx.x; k < s; k += blockDim.x) {
                double tv = a_of(k) * pc[k];
                if (k > 0) tv += b_of(k) * pc[k - 1];
                if (k + 1 < s) tv += b_of(k + 1) * pc[k + 1];
                pn[k] = 2.0 * (pc[k] - g * tv) - pp[k];
                u[k] += cc.d[j] * pn[k];
            }
            __syncthreads();
            double *t = pp; pp = pc; pc = pn; pn = t;
        }
    } else {
        const QuadRule &q = tc.q;
        if (q.n > 0) {
            // fractional factor: u = sum_j W_j (sigma_j I + T)^{-1} e_1, one node per thread
            // (Thomas algorithm: modified super-diagonal in cq, solution in xq), then the
            // weighted sum per row in a fixed order
            double *qw = qwork + int64_t(c) * 2 * m * q.n;
            for (int j = threadIdx.x; j < q.n; j += blockDim.x) {
                double *cq = qw + int64_t(j) * 2 * m, *xq = cq + m;
                const double sg = q.shift[j];
                double piv = 1.0 / (sg + a_of(0));
                cq[0] = (s > 1) ? b_of(1) * piv : 0.0;
                xq[0] = piv;
                for (int k = 1; k < s; ++k) {
                    piv = 1.0 / (sg + a_of(k) - b_of(k) * cq[k - 1]);
                    cq[k] = (k + 1 < s) ? b_of(k + 1) * piv : 0.0;
                    xq[k] = -b_of(k) * xq[k - 1] * piv;
                }
                for (int k = s - 2; k >= 0; --k) xq[k] -= cq[k] * xq[k + 1];
            }
            __syncthreads();
            for (int k = threadIdx.x; k < s; k += blockDim.x) {
                double acc = 0.0;
                for (int j = 0; j < q.n; ++j) acc = fma(q.weight[j], qw[int64_t(j) * 2 * m + m + k], acc);
                u[k] = acc;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            // (eps I + T) = L U: v0 = modified super-diagonal, v2 = reciprocal pivots (once);
            // then s_int forward / backward sweeps from rhs = e_1 (or from the fractional factor)
            double den = eps + a_of(0);
            v2[0] = 1.0 / den;
            v0[0] = (s > 1) ? b_of(1) * v2[0] : 0.0;
            for (int k = 1; k < s; ++k) {
                den = eps + a_of(k) - b_of(k) * v0[k - 1];
                v2[k] = 1.0 / den;
                v0[k] = (k + 1 < s) ? b_of(k + 1) * v2[k] : 0.0;
            }
            if (q.n == 0) u[0] = 1.0;
            for (int rep = 0; rep < s_int; ++rep) {
                v1[0] = u[0] * v2[0];
                for (int k = 1; k < s; ++k) v1[k] = (u[k] - b_of(k) * v1[k - 1]) * v2[k];
                u[s - 1] = v1[s - 1];
                for (int k = s - 2; k >= 0; --k) u[k] = v1[k] - v0[k] * u[k + 1];
            }
        }
    }
    __syncthreads();
    // phi(T) e_1 within max phi on [0, Lambda] unless T left the interval (lost orthogonality)
    {
        bool bad = false;
        for (int k = threadIdx.x; k < s; k += blockDim.x)
            if (!(fabs(u[k]) <= bound)) bad = true;
        if (__syncthreads_or(bad) && threadIdx.x == 0)
            atomicCAS(reinterpret_cast<int *>(&ctrl->status), KB_OK, KB_ERR_ORTHOGONALITY);
    }
    // E_W = P_1 and Q_1 = sigma_1 P_1, so Y = (1/sigma_1) [Q_1..Q_m] phi(T) e_1
    // (the sqrt(N) factor of Algorithm 2's final step, for the global method)
    const double scale = 1.0 / sigma[c];
    if (gbl) {
        for (int idx = threadIdx.x; idx < m * W; idx += blockDim.x) {
            const int k = idx / W, c2 = idx % W;
            omega[idx] = (c2 < M && k < s) ? scale * u[k] * sigma[int64_t(k) * W] : 0.0;
        }
    } else {
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            omega[int64_t(k) * W + c] = k < s ? scale * u[k] * sigma[int64_t(k) * W + c] : 0.0;
    }
}

// X[:, c] -= a[c] * P[:, c]; partial column sums of X^2 per CTA.  Rows of tiles beyond
// the frontier limit are zero in X and P and are skipped.
template <typename T, int W>
__global__ void __launch_bounds__(256) k_axpy_colnorm(T *X, const T *P, const double *a, int64_t n,
                                                       double *parts, const Ctrl *ctrl,
                                                       const int32_t *tgen, int limit,
                                                       const int32_t *alist, const int32_t *acount,
                                                       ProfCount pc) {
    if (ctrl->stop) return;
    using C = typename Cmp<T>::type;
    constexpr int CG = W / 4;
    constexpr int RPP = 256 / CG;   // rows per pass
    __shared__ double s[RPP][W];
    const int cg = threadIdx.x % CG, rr = threadIdx.x / CG;
    const int c4 = cg * 4;
    C ah[4], al[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        ah[q] = C(a[c4 + q]);
        al[q] = C(a[c4 + q] - double(ah[q]));
    }
    C acc[4] = {0, 0, 0, 0};
    unsigned long long my_rows = 0;
    if (alist && tgen) {
        // active 32-row tiles only (listed in increasing order): RPP rows per pass
        const int cnt = *acount;
        for (int it = blockIdx.x; it < cnt; it += gridDim.x) {
            const int64_t t0 = int64_t(__ldg(alist + it)) * ACT_ROWS;
            for (int sub = rr; sub < ACT_ROWS; sub += RPP) {
                const int64_t row = t0 + sub;
                if (row >= n) break;
                C xv[4], pv[4];
                ldv4(X + row * W + c4, xv);
                ldv4(P + row * W + c4, pv);
                if (cg == 0) ++my_rows;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    xv[q] = xv[q] - fma(ah[q], pv[q], al[q] * pv[q]);
                    if constexpr (!std::is_same<T, C>::value) xv[q] = C(T(xv[q]));
                    acc[q] = fma(xv[q], xv[q], acc[q]);
                }
                stv4(X + row * W + c4, xv);
            }
        }
    }
    // two rows per iteration, 16-byte vector accesses: four loads in flight per thread
    const int64_t stride = int64_t(gridDim.x) * RPP;
    for (int64_t row = int64_t(blockIdx.x) * RPP + rr; !(alist && tgen) && row < n; row += 2 * stride) {
        const int64_t row2 = row + stride;
        const bool act0 = !tgen || __ldg(tgen + row / ACT_ROWS) <= limit;
        const bool act1 = row2 < n && (!tgen || __ldg(tgen + row2 / ACT_ROWS) <= limit);
        C xv[2][4], pv[2][4];
        if (act0) {
            ldv4(X + row * W + c4, xv[0]);
            ldv4(P + row * W + c4, pv[0]);
        }
        if (act1) {
            ldv4(X + row2 * W + c4, xv[1]);
            ldv4(P + row2 * W + c4, pv[1]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!(h ? act1 : act0)) continue;
            if (cg == 0) ++my_rows;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                xv[h][q] = xv[h][q] - fma(ah[q], pv[h][q], al[q] * pv[h][q]);
                // the norm is that of the stored (narrowed) value
                if constexpr (!std::is_same<T, C>::value) xv[h][q] = C(T(xv[h][q]));
                acc[q] = fma(xv[h][q], xv[h][q], acc[q]);
            }
            stv4(X + (h ? row2 : row) * W + c4, xv[h]);
        }
    }
    if (pc.rows && cg == 0 && my_rows) atomicAdd(pc.rows, my_rows);
    if constexpr (std::is_same<C, float>::value) {
        // double-float column sums on the FP32 pipe; partials written as DF pairs
        DF *sd = reinterpret_cast<DF *>(&s[0][0]);
#pragma unroll
        for (int q = 0; q < 4; ++q) sd[rr * W + c4 + q] = DF{acc[q], 0.f};
        __syncthreads();
        DF *out = reinterpret_cast<DF *>(parts);
        for (int c = threadIdx.x; c < W; c += 256) {
            DF t = sd[c];
            for (int r = 1; r < RPP; ++r) df_merge(t, sd[r * W + c]);
            out[int64_t(blockIdx.x) * W + c] = t;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) s[rr][c4 + q] = acc[q];
        __syncthreads();
        for (int c = threadIdx.x; c < W; c += 256) {
            double t = 0.0;
            for (int r = 0; r < RPP; ++r) t += s[r][c];
            parts[int64_t(blockIdx.x) * W + c] = t;
        }
    }
}

// Y[i, c] = sum_k omega_k[c] P_k[i, c]  (global / sequential Lanczos assembly); with a
// frontier, block kbase + k is zero in rows whose tile is more than kbase + k hops from W.
// accumulate: Y is added to (the FP32 accumulator starts from Y, so adding the blocks one
// launch at a time gives the same bits as one launch over all of them).
template <typename T, int W>
__global__ void __launch_bounds__(256) k_assemble_diag(const T *basis, int64_t stride, int nblk,
                                                        const double *omega, int64_t n, float *Y,
                                                        int64_t ldy, int mo, const int32_t *tgen,
                                                        int kbase, int accumulate, ProfCount pc) {
    constexpr int CG = W / 4;
    constexpr int RPP = 256 / CG;
    using C = typename Cmp<T>::type;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C *som = reinterpret_cast<C *>(sm_raw);     // [nblk][W]
    for (int i = threadIdx.x; i < nblk * W; i += blockDim.x) som[i] = C(omega[i]);
    __syncthreads();
    const int cg = threadIdx.x % CG, rr = threadIdx.x / CG;
    const int c4 = cg * 4;
    unsigned long long my_units = 0;
    for (int64_t row = int64_t(blockIdx.x) * RPP + rr; row < n; row += int64_t(gridDim.x) * RPP) {
        C acc[4] = {0, 0, 0, 0};
        if (accumulate)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (c4 + q < mo) acc[q] = Y[row * ldy + c4 + q];
        const int k0 = tgen ? min(max(__ldg(tgen + row / ACT_ROWS) - kbase, 0), nblk) : 0;
        if (cg == 0) my_units += nblk - k0;
        for (int k = k0; k < nblk; ++k) {
            C pv[4];
            ldv4(basis + int64_t(k) * stride + row * W + c4, pv);
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(som[k * W + c4 + q], pv[q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (c4 + q < mo) Y[row * ldy + c4 + q] = acc[q];
    }
    if (pc.nnz && cg == 0 && my_units) atomicAdd(pc.nnz, my_units);
}

// ---------------------------------------------------------------- frontier
__global__ void k_frontier_seed(uint8_t *gen, int32_t *tgen, NodeChunk ch) {
    const int j = threadIdx.x + blockIdx.x * blockDim.x;
    if (j < ch.cnt) {
        gen[ch.idx[j]] = 0;
        tgen[ch.idx[j] / ACT_ROWS] = 0;
    }
}

// One hop: rows at distance k-1 mark their unreached neighbours with distance k.
// Marks the unreached neighbours of one frontier row (stored nonzeros beg..end) with
// distance k, eight at a time: their indices, then their marks, loaded before any store (a
// mark read as unset that another thread sets meanwhile only repeats the same store).
__device__ __forceinline__ void expand_row(const GraphDev &g, uint8_t *gen, int32_t *tgen, int k,
                                           int beg, int end) {
    for (int p = beg; p < end; p += 8) {
        int jj[8];
        uint8_t gj[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) jj[u] = p + u < end ? __ldg(g.col + p + u) : -1;
#pragma unroll
        for (int u = 0; u < 8; ++u) gj[u] = jj[u] >= 0 ? gen[jj[u]] : uint8_t(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (gj[u] == 255) {
                gen[jj[u]] = uint8_t(k);
                atomicMin(tgen + jj[u] / ACT_ROWS, k);
            }
    }
}

__global__ void __launch_bounds__(256) k_frontier_expand(GraphDev g, uint8_t *gen, int32_t *tgen, int k) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.n;
         i += int64_t(gridDim.x) * blockDim.x) {
        if (__ldg(tgen + i / ACT_ROWS) > k - 1) continue;
        if (gen[i] != uint8_t(k - 1)) continue;
        const int beg = __ldg(g.rowptr + i), end = __ldg(g.rowptr + i + 1);
        expand_row(g, gen, tgen, k, beg, end);
    }
}

template <typename T>
__global__ void k_u_convert(const double *U, int M, int W, int m, T *Ut, const Ctrl *ctrl) {
    // U: (steps*M) x M row-major -> Ut: (m*W) x W, zero padded, zero beyond steps
    const int steps = ctrl->steps;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < int64_t(m) * W * W;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int blk = int(idx / (W * W));
        const int i = int((idx / W) % W), j = int(idx % W);
        double v = 0.0;
        if (blk < steps && i < M && j < M) v = U[(int64_t(blk) * M + i) * M + j];
        Ut[idx] = T(v);
    }
}

// phi(H) F_1 (or phi(T) e_1) must stay within the bound that holds when the projected
// matrix has its spectrum in [0, Lambda]; a NaN or a larger entry means the Lanczos basis
// lost orthogonality, and the solve is marked KB_ERR_ORTHOGONALITY (Y is then NaN-filled).
__global__ void k_check_projected(const double *U, int64_t count, double bound, Ctrl *ctrl) {
    if (ctrl->status != KB_OK) return;
    bool bad = false;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x)
        if (!(fabs(U[i]) <= bound)) bad = true;
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicCAS(reinterpret_cast<int *>(&ctrl->status), KB_OK, KB_ERR_ORTHOGONALITY);
}

// ---------------------------------------------------------------- launchers
int launch_check_projected(const double *U, int64_t count, double bound, Ctrl *ctrl, cudaStream_t s) {
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, int64_t(num_sms()) * 2)));
    k_check_projected<<<grid, 256, 0, s>>>(U, count, bound, ctrl);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

namespace {
__global__ void k_ctrl_snapshot(Ctrl *dst, const Ctrl *src, int k) {
    Ctrl c = *src;
    // once the process stopped (converged, invariant space, breakdown) later checks have
    // nothing to decide: zero steps make the projected kernels return at once
    c.steps = src->stop ? 0 : min(c.steps, k);
    c.stop = 0;
    *dst = c;
}

__global__ void __launch_bounds__(1024) k_conv_check(const double *U, const double *Up, int M,
                                                     const Ctrl *chk, int32_t *prev_steps,
                                                     double tol, Ctrl *ctrl, int buf) {
    if (ctrl->stop) return;   // already stopped (invariant space, breakdown or converged)
    __shared__ double sd[32], sn[32];
    const int steps = chk->steps, ps = *prev_steps;
    const int64_t cnt = int64_t(steps) * M * M, pcnt = int64_t(ps) * M * M;
    double d2 = 0.0, n2 = 0.0;
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const double u = U[i];
        const double e = u - (i < pcnt ? Up[i] : 0.0);
        d2 = fma(e, e, d2);
        n2 = fma(u, u, n2);
    }
    for (int off = 16; off > 0; off >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, off);
        n2 += __shfl_xor_sync(0xffffffffu, n2, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sd[warp] = d2; sn[warp] = n2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double D = 0.0, N = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) { D += sd[w]; N += sn[w]; }
        if (ps > 0) {
            const double change = N > 0.0 ? sqrt(D) / sqrt(N) : 0.0;
            ctrl->est_change = change;
            if (change <= tol) {
                ctrl->stop = 1;
                ctrl->steps = steps;
                ctrl->from_check = buf;   // U of this check is the result: no second solve
            }
        }
        *prev_steps = steps;
    }
}
}  // namespace

int launch_ctrl_snapshot(Ctrl *dst, const Ctrl *src, int k, cudaStream_t s) {
    k_ctrl_snapshot<<<1, 1, 0, s>>>(dst, src, k);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

// The control block the final projected solve runs on: a copy of ctrl with no steps when
// the stopping rule already formed U at its last check (then k_copy_check_u supplies it).
__global__ void k_ctrl_final(Ctrl *dst, const Ctrl *src) {
    Ctrl c = *src;
    if (c.from_check >= 0) c.steps = 0;
    *dst = c;
}
__global__ void k_copy_check_u(const double *Uc, int64_t per, double *U, int M, const Ctrl *ctrl) {
    const int b = ctrl->from_check;
    if (b < 0) return;
    (void)M;
    const int64_t cnt = per;   // the check zeroed its whole buffer: copy it all
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < cnt; i += int64_t(gridDim.x) * blockDim.x)
        U[i] = Uc[b * per + i];
}
int launch_ctrl_final(Ctrl *dst, const Ctrl *src, cudaStream_t s) {
    k_ctrl_final<<<1, 1, 0, s>>>(dst, src);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}
int launch_copy_check_u(const double *Uc, int64_t per, double *U, int M, int m, const Ctrl *ctrl,
                        cudaStream_t s) {
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>((int64_t(m) * M * M + 255) / 256, 4 * int64_t(num_sms()))));
    k_copy_check_u<<<grid, 256, 0, s>>>(Uc, per, U, M, ctrl);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

int launch_conv_check(const double *U, const double *Up, int M, const Ctrl *chk, int32_t *prev_steps,
                      double tol, Ctrl *ctrl, cudaStream_t s, int buf) {
    prof_begin(KernelClass::SMALL, s);
    k_conv_check<<<1, 1024, 0, s>>>(U, Up, M, chk, prev_steps, tol, ctrl, buf);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::SMALL, s, 0, 0);
    return 0;
}

int launch_ctrl_init(Ctrl *c, int steps, cudaStream_t s) {
    k_ctrl_init<<<1, 1, 0, s>>>(c, steps);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "k_ctrl_init");
}

template <typename T>
int launch_scatter(T *block, int64_t ld, const int32_t *nodes, int M, int col0, T val, cudaStream_t s) {
    for (int j0 = 0; j0 < M; j0 += NodeChunk::CAP) {
        NodeChunk ch;
        ch.cnt = std::min(NodeChunk::CAP, M - j0);
        ch.col0 = col0 + j0;
        for (int j = 0; j < ch.cnt; ++j) ch.idx[j] = nodes[j0 + j];
        k_scatter<T><<<1, NodeChunk::CAP, 0, s>>>(block, ld, ch, val);
        count_launches(1);
    }
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

int launch_marker(int32_t *marker, const int32_t *nodes, int M, cudaStream_t s) {
    for (int j0 = 0; j0 < M; j0 += NodeChunk::CAP) {
        NodeChunk ch;
        ch.cnt = std::min(NodeChunk::CAP, M - j0);
        ch.col0 = j0;
        for (int j = 0; j < ch.cnt; ++j) ch.idx[j] = nodes[j0 + j];
        k_marker<<<1, NodeChunk::CAP, 0, s>>>(marker, ch);
        count_launches(1);
    }
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

template <typename T>
int launch_scale_copy(T *out, const T *in, int64_t count, double scale, cudaStream_t s) {
    const int grid = int(std::min<int64_t>((count + 255) / 256, int64_t(num_sms()) * 8));
    k_scale_copy<T><<<std::max(grid, 1), 256, 0, s>>>(out, in, count, scale);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

int launch_frontier_init(uint8_t *gen, int32_t *tgen, int64_t n, const int32_t *nodes, int M,
                         cudaStream_t s) {
    KB_CUDA_TRY(cudaMemsetAsync(gen, 0xFF, size_t(n), s));
    KB_CUDA_TRY(cudaMemsetAsync(tgen, 0x7F, sizeof(int32_t) * size_t((n + ACT_ROWS - 1) / ACT_ROWS), s));
    for (int j0 = 0; j0 < M; j0 += NodeChunk::CAP) {
        NodeChunk ch;
        ch.cnt = std::min(NodeChunk::CAP, M - j0);
        ch.col0 = j0;
        for (int j = 0; j < ch.cnt; ++j) ch.idx[j] = nodes[j0 + j];
        k_frontier_seed<<<1, NodeChunk::CAP, 0, s>>>(gen, tgen, ch);
        count_launches(1);
    }
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

// Same as k_frontier_expand, visiting only the rows of the 32-row tiles active at step k-1
// (the list made after the previous expansion): the rows at distance k-1 lie there.
__global__ void __launch_bounds__(256) k_frontier_expand_listed(GraphDev g, uint8_t *gen, int32_t *tgen, int k,
                                                                const int32_t *__restrict__ alist,
                                                                const int32_t *__restrict__ acount) {
    const int64_t total = int64_t(*acount) * ACT_ROWS;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = int64_t(__ldg(alist + idx / ACT_ROWS)) * ACT_ROWS + idx % ACT_ROWS;
        if (i >= g.n || gen[i] != uint8_t(k - 1)) continue;
        const int beg = __ldg(g.rowptr + i), end = __ldg(g.rowptr + i + 1);
        expand_row(g, gen, tgen, k, beg, end);
    }
}

// Stream compaction of the active 32-row tiles in tile order.  Each warp owns a contiguous
// range of 32-entry groups and reads them coalesced, eight groups in flight; a ballot gives
// each group's active lanes, kept in shared memory (up to LIST_MASKS groups, i.e. 2^18 tiles
// of 32 rows; beyond that the second pass reads the array again).  The warp's count and, in
// the second pass, each active entry's position (the active lanes below it) come from
// population counts; a block-wide exclusive scan of the warp counts gives each warp's offset.
constexpr int LIST_MASKS = 8192;
__global__ void __launch_bounds__(1024) k_frontier_list(const int32_t *__restrict__ tgen, int64_t nact,
                                                        int limit, int32_t *__restrict__ list,
                                                        int32_t *__restrict__ count) {
    __shared__ int wsum[33];
    __shared__ unsigned s_mask[LIST_MASKS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t ngrp = (nact + 31) / 32;
    const bool cached = ngrp <= LIST_MASKS;
    const int64_t gper = (ngrp + nw - 1) / nw;
    const int64_t g0 = int64_t(warp) * gper;
    const int64_t g1 = g0 + gper < ngrp ? g0 + gper : ngrp;
    int c = 0;
    for (int64_t g = g0; g < g1; g += 8) {
        int32_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t a = (g + u) * 32 + lane;
            v[u] = (g + u < g1 && a < nact) ? __ldg(tgen + a) : INT_MAX;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const unsigned mask = __ballot_sync(0xffffffffu, v[u] <= limit);
            if (cached && lane == 0 && g + u < g1) s_mask[g + u] = mask;
            c += __popc(mask);
        }
    }
    if (lane == 0) wsum[warp] = c;
    __syncthreads();
    if (warp == 0) {
        const int own = lane < nw ? wsum[lane] : 0;
        int incl = own;
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += u;
        }
        wsum[lane] = incl - own;               // exclusive offset of warp `lane`
        if (lane == 31) wsum[32] = incl;       // total
    }
    __syncthreads();
    int pos = wsum[warp];
    const unsigned below = (1u << lane) - 1u;
    for (int64_t g = g0; g < g1; g += 8) {
        unsigned mk[8];
        if (cached) {
#pragma unroll
            for (int u = 0; u < 8; ++u) mk[u] = g + u < g1 ? s_mask[g + u] : 0u;
        } else {
            int32_t v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t a = (g + u) * 32 + lane;
                v[u] = (g + u < g1 && a < nact) ? __ldg(tgen + a) : INT_MAX;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) mk[u] = __ballot_sync(0xffffffffu, v[u] <= limit);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if ((mk[u] >> lane) & 1u) list[pos + __popc(mk[u] & below)] = int32_t((g + u) * 32 + lane);
            pos += __popc(mk[u]);
        }
    }
    if (threadIdx.x == 0) *count = wsum[32];
}

int launch_frontier_list(const int32_t *tgen, int64_t n, int limit, int32_t *list, int32_t *count,
                         cudaStream_t s) {
    prof_begin(KernelClass::OTHER, s);
    k_frontier_list<<<1, 1024, 0, s>>>(tgen, (n + ACT_ROWS - 1) / ACT_ROWS, limit, list, count);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::OTHER, s, double(n) / ACT_ROWS * 4, 0);
    return 0;
}

int launch_frontier_expand(const GraphDev &g, uint8_t *gen, int32_t *tgen, int k, cudaStream_t s,
                           const int32_t *alist, const int32_t *acount) {
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>((g.n + 255) / 256, int64_t(num_sms()) * 8)));
    prof_begin(KernelClass::OTHER, s);
    if (alist) k_frontier_expand_listed<<<grid, 256, 0, s>>>(g, gen, tgen, k, alist, acount);
    else k_frontier_expand<<<grid, 256, 0, s>>>(g, gen, tgen, k);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::OTHER, s, double(g.n) / ACT_ROWS * 4, 0);
    return 0;
}

int launch_fill_nan(float *Y, int64_t n, int64_t ldy, int mo, const Ctrl *ctrl, cudaStream_t s) {
    const int grid = int(std::min<int64_t>((n * mo + 255) / 256, int64_t(num_sms()) * 8));
    k_fill_nan<<<std::max(grid, 1), 256, 0, s>>>(Y, n, ldy, mo, ctrl);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

template <typename T>
int launch_hkk(const double *G, int M, int W, double *Hd, T *C, const Ctrl *ctrl, cudaStream_t s) {
    prof_begin(KernelClass::SMALL, s);
    k_hkk<T><<<1, 1024, 0, s>>>(G, M, W, Hd, C, ctrl);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::SMALL, s, 0, 0);
    return 0;
}

template <typename T>
int launch_chol(const double *G, int M, int W, int pass, int step, double inv_thresh2,
                double piv_rel2, double *R1, T *Rinv, double *Hs, T *Bout, Ctrl *ctrl,
                cudaStream_t s) {
    auto bytes_for = [](int m) {
        const bool newton = sizeof(T) == 4 && m <= CHOL_NEWTON_MAX;
        return sizeof(double) * size_t(m) * (m + 1) + sizeof(T) * (size_t(m) * (m + 1) + 2) +
               sizeof(double) * size_t(3 * m + 2) +
               (newton ? (sizeof(double) + 2 * sizeof(float)) * size_t(m) * (m + 1) : 0) +
               sizeof(T) * size_t(tri_inv_tmp_elems(m));
    };
    const size_t smem = bytes_for(M);
    // FP64 blocks are at most 64 wide; function-local static: set once, thread-safe
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_chol<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes_for(sizeof(T) == 8 ? 64 : 128)));
    (void)attr;
    prof_begin(KernelClass::SMALL, s);
    k_chol<T><<<1, 256, smem, s>>>(G, M, W, pass, step, inv_thresh2, piv_rel2, R1, Rinv, Hs,
                                   Bout, ctrl);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::SMALL, s, 0, 0);
    return 0;
}

int launch_lanczos_init(int W, int M, int gbl, int round32, double *sigma, int32_t *alive,
                        double *c1, double *c2, cudaStream_t s) {
    k_lanczos_init<<<1, 128, 0, s>>>(W, M, gbl, round32, sigma, alive, c1, c2);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

int launch_lanczos_alpha(const double *parts, int nparts, int W, int M, int gbl, int k, int df,
                         const double *sigma, double *alpha, double *a_upd, const Ctrl *ctrl,
                         cudaStream_t s) {
    prof_begin(KernelClass::SMALL, s);
    k_lanczos_alpha<<<1, 1024, 0, s>>>(parts, nparts, W, M, gbl, k, df, sigma, alpha, a_upd, ctrl);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::SMALL, s, double(nparts) * W * 8, 0);
    return 0;
}

int launch_lanczos_beta(const double *parts, int nparts, int W, int M, int gbl, int k, int round32,
                        double thresh, double *beta, double *sigma, int32_t *alive, double *c1,
                        double *c2, Ctrl *ctrl, cudaStream_t s) {
    prof_begin(KernelClass::SMALL, s);
    k_lanczos_beta<<<1, 1024, 0, s>>>(parts, nparts, W, M, gbl, k, round32, thresh, beta, sigma,
                                     alive, c1, c2, ctrl);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::SMALL, s, double(nparts) * W * 8, 0);
    return 0;
}

int launch_tridiag_phi(int W, int M, int m, int gbl, const double *alpha, const double *beta,
                       const double *sigma, int phi_kind, double eps, int s_int, double lam,
                       const TriCoef &tc, double *omega, double *work, double *qwork, Ctrl *ctrl,
                       double bound, cudaStream_t s, const std::vector<double> *series) {
    prof_begin(KernelClass::PROJECTED, s);
    int launches = 1, u_ready = 0;
    if (phi_kind == KB_PHI_EXP && series && int(series->size()) > ChebCoef::CAP) {
        // a series longer than one parameter block: chunks of CAP terms, state in work
        for (size_t j0 = 0; j0 < series->size(); j0 += ChebCoef::CAP) {
            ChebCoef cc{};
            cc.n = int(std::min<size_t>(ChebCoef::CAP, series->size() - j0));
            for (int q = 0; q < cc.n; ++q) cc.d[q] = (*series)[j0 + q];
            k_tridiag_exp_chunk<<<gbl ? 1 : W, TRI_THREADS, 0, s>>>(W, M, m, gbl, alpha, beta, lam, cc,
                                                                    int(j0), work, ctrl);
            ++launches;
        }
        u_ready = 1;
    }
    const size_t smem = (m <= TRI_SMEM_M && !u_ready) ? sizeof(double) * 6 * size_t(m) : 0;
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_tridiag_phi, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(double) * 6 * TRI_SMEM_M));
    (void)attr;
    k_tridiag_phi<<<gbl ? 1 : W, TRI_THREADS, smem, s>>>(W, M, m, gbl, alpha, beta, sigma,
                                                         phi_kind, eps, s_int, lam, tc, omega,
                                                         work, qwork, ctrl, bound, u_ready);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::PROJECTED, s, 0, 0, launches);
    return 0;
}

template <typename T>
int launch_axpy_colnorm(int W, T *X, const T *P, const double *a, int64_t n, double *parts,
                        int *grid_out, const Ctrl *ctrl, const int32_t *tgen, int limit,
                        int64_t M_alg, cudaStream_t s, const int32_t *alist, const int32_t *acount) {
    const int rpp = 256 / (W / 4);
    const int grid = int(std::min<int64_t>((n + rpp - 1) / rpp, int64_t(num_sms()) * 4));
    *grid_out = std::max(grid, 1);
    const ProfCount pc = prof_begin(KernelClass::ROWBLOCK, s);
    switch (W) {
        case 16: k_axpy_colnorm<T, 16><<<*grid_out, 256, 0, s>>>(X, P, a, n, parts, ctrl, tgen, limit, alist, acount, pc); break;
        case 32: k_axpy_colnorm<T, 32><<<*grid_out, 256, 0, s>>>(X, P, a, n, parts, ctrl, tgen, limit, alist, acount, pc); break;
        case 64: k_axpy_colnorm<T, 64><<<*grid_out, 256, 0, s>>>(X, P, a, n, parts, ctrl, tgen, limit, alist, acount, pc); break;
        case 128: k_axpy_colnorm<T, 128><<<*grid_out, 256, 0, s>>>(X, P, a, n, parts, ctrl, tgen, limit, alist, acount, pc); break;
        default: return fail(KB_ERR_ARG, "bad width");
    }
    KB_CUDA_TRY(cudaGetLastError());
    const double row = double(M_alg) * sizeof(T);
    prof_end(KernelClass::ROWBLOCK, s, 3.0 * double(n) * row, 3.0 * double(n) * M_alg, 1, 3.0 * row,
             0.0, 3.0 * M_alg, 0.0);
    return 0;
}

int axpy_max_grid() { return num_sms() * 4; }

#define KB_ASM_DIAG(WW)                                                                       \
    do {                                                                                      \
        cudaFuncSetAttribute(k_assemble_diag<T, WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             int(smem));                                                      \
        k_assemble_diag<T, WW><<<grid, 256, smem, s>>>(basis, stride, nblk, omega, n, Y, ldy, mo,  \
                                                       tgen, kbase, accumulate, pc);          \
    } while (0)

template <typename T>
int launch_assemble_diag(int W, const T *basis, int64_t stride, int nblk, const double *omega,
                         int64_t n, float *Y, int64_t ldy, int mo, int64_t M_alg,
                         const int32_t *tgen, cudaStream_t s, int kbase, int accumulate) {
    const int rpp = 256 / (W / 4);
    const int grid = std::max(1, int(std::min<int64_t>((n + rpp - 1) / rpp, int64_t(num_sms()) * 8)));
    const size_t smem = sizeof(typename Cmp<T>::type) * size_t(nblk) * W;
    if (smem > 200 * 1024) return fail(KB_ERR_UNSUPPORTED, "too many blocks for the diagonal assembly");
    const ProfCount pc = prof_begin(KernelClass::ASSEMBLE, s);
    switch (W) {
        case 16: KB_ASM_DIAG(16); break;
        case 32: KB_ASM_DIAG(32); break;
        case 64: KB_ASM_DIAG(64); break;
        case 128: KB_ASM_DIAG(128); break;
        default: return fail(KB_ERR_ARG, "bad width");
    }
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::ASSEMBLE, s, double(nblk) * n * M_alg * sizeof(T) + double(n) * M_alg * 4,
             2.0 * nblk * double(n) * M_alg, 1, 0.0, double(M_alg) * sizeof(T), 0.0,
             double(n) * M_alg * 4);
    return 0;
}

template <typename T>
int launch_u_convert(const double *U, int M, int W, int m, T *Ut, const Ctrl *ctrl, cudaStream_t s) {
    const int64_t cnt = int64_t(m) * W * W;
    const int grid = int(std::min<int64_t>((cnt + 255) / 256, 1024));
    k_u_convert<T><<<std::max(grid, 1), 256, 0, s>>>(U, M, W, m, Ut, ctrl);
    count_launches(1);
    KB_CUDA_TRY(cudaGetLastError());
    return 0;
}

#define KB_INST(T)                                                                              \
    template int launch_scatter<T>(T *, int64_t, const int32_t *, int, int, T, cudaStream_t);   \
    template int launch_scale_copy<T>(T *, const T *, int64_t, double, cudaStream_t);           \
    template int launch_hkk<T>(const double *, int, int, double *, T *, const Ctrl *, cudaStream_t); \
    template int launch_chol<T>(const double *, int, int, int, int, double, double, double *,   \
                                T *, double *, T *, Ctrl *, cudaStream_t);                      \
    template int launch_axpy_colnorm<T>(int, T *, const T *, const double *, int64_t, double *,  \
                                        int *, const Ctrl *, const int32_t *, int, int64_t,     \
                                        cudaStream_t, const int32_t *, const int32_t *);        \
    template int launch_assemble_diag<T>(int, const T *, int64_t, int, const double *, int64_t, \
                                         float *, int64_t, int, int64_t, const int32_t *,       \
                                         cudaStream_t, int, int);                               \
    template int launch_u_convert<T>(const double *, int, int, int, T *, const Ctrl *, cudaStream_t);
KB_INST(float)
KB_INST(double)
#undef KB_INST
// BF16 blocks: element-wise kernels on the stored type (small matrices stay FP32)
template int launch_scatter<__nv_bfloat16>(__nv_bfloat16 *, int64_t, const int32_t *, int, int,
                                           __nv_bfloat16, cudaStream_t);
template int launch_scale_copy<__nv_bfloat16>(__nv_bfloat16 *, const __nv_bfloat16 *, int64_t,
                                              double, cudaStream_t);
template int launch_axpy_colnorm<__nv_bfloat16>(int, __nv_bfloat16 *, const __nv_bfloat16 *,
                                                const double *, int64_t, double *, int *,
                                                const Ctrl *, const int32_t *, int, int64_t,
                                                cudaStream_t, const int32_t *, const int32_t *);
template int launch_assemble_diag<__nv_bfloat16>(int, const __nv_bfloat16 *, int64_t, int,
                                                 const double *, int64_t, float *, int64_t, int,
                                                 int64_t, const int32_t *, cudaStream_t, int, int);

}  // namespace kb
