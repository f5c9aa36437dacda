// The projected problem U = phi(H_m) F_1 of the classical block Lanczos method
// (the projected step of Algorithm 1), in FP64 on the device.
//
// H_m is block tridiagonal: diagonal blocks H_kk (symmetric) and sub-diagonal blocks
// H_{k+1,k} = R (upper triangular), super-diagonal blocks R^T.  Its spectrum lies in
// [0, Lambda] (interlacing, proof of Theorem 3.1), so:
//   * exp:    U = sum_j d_j T_j(I - 2 H/Lambda) F_1 with the Chebyshev coefficients d_j
//             of e^{-t lambda} on [0, Lambda] (computed on the host from modified Bessel
//             functions), by the three-term recurrence on the block vectors V_j.  V_j is
//             supported on block rows 0..j, so iteration j touches only j+2 block rows.
//   * spline: for integer s, s solves with the SPD block tridiagonal eps I + H_m through
//             its block Cholesky factorisation (block Thomas algorithm).  For non-integer s
//             the fractional factor (eps I + H_m)^{-alpha} F_1 is the quadrature sum
//             sum_k W_k (sigma_k I + H_m)^{-1} F_1 over real shifts sigma_k > eps
//             (quadrature.cu), one block Cholesky factorisation and solve per node, the nodes
//             in parallel (one CTA each), followed by floor(s) solves with eps I + H_m.
// Both give the same U as the spectral evaluation assumed in Section 7, up to FP64
// rounding (the Chebyshev series is truncated below 1e-17 relative).
#include "kb_internal.cuh"
#include "kb_kernels.cuh"

namespace kb {
namespace {

constexpr int TC = 4;    // output columns per CTA (many small CTAs: the FP64 work spreads over all SMs)

// U = 0, only when the solve has steps: the stopping rule's later checks run with no steps
// and must leave the buffer of the check that stopped the process as it is.
__global__ void k_zero_if_active(double *U, int64_t count, const Ctrl *ctrl) {
    if (ctrl->steps <= 0) return;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x)
        U[i] = 0.0;
}
int zero_if_active(double *U, int64_t count, const Ctrl *ctrl, cudaStream_t s) {
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 4 * int64_t(num_sms()))));
    k_zero_if_active<<<grid, 256, 0, s>>>(U, count, ctrl);
    return 0;
}

__global__ void k_cheb_bt_seed(double *V0, double *U, int M, double d0, const Ctrl *ctrl) {
    const int i = threadIdx.x + blockIdx.x * blockDim.x;
    if (ctrl->steps > 0 && i < M) {
        V0[int64_t(i) * M + i] = 1.0;
        U[int64_t(i) * M + i] = d0;
    }
}

// V_{j+1} = beta (V_j - g H V_j) - gamma V_{j-1};  U += d_{j+1} V_{j+1}
__global__ void __launch_bounds__(256)
k_cheb_bt_iter(const double *__restrict__ Hd, const double *__restrict__ Hs,
               const double *__restrict__ Vp, const double *__restrict__ Vc, double *__restrict__ Vn,
               double *__restrict__ U, int M, double beta, double gamma, double dnext, double g,
               const Ctrl *ctrl) {
    const int r = blockIdx.x;
    const int steps = ctrl->steps;
    if (r >= steps) return;
    const int c0 = blockIdx.y * TC;
    extern __shared__ double sv[];   // [3][M][TC]
    double *s0 = sv, *s1 = sv + M * TC, *s2 = sv + 2 * M * TC;
    const int64_t MM = int64_t(M) * M;
    for (int idx = threadIdx.x; idx < M * TC; idx += blockDim.x) {
        const int k = idx / TC, cc = idx % TC, c = c0 + cc;
        double a = 0.0, b = 0.0, d = 0.0;
        if (c < M) {
            if (r > 0) a = Vc[(r - 1) * MM + int64_t(k) * M + c];
            b = Vc[r * MM + int64_t(k) * M + c];
            if (r + 1 < steps) d = Vc[(r + 1) * MM + int64_t(k) * M + c];
        }
        s0[idx] = a; s1[idx] = b; s2[idx] = d;
    }
    __syncthreads();
    const double *hd = Hd + r * MM;
    const double *hl = (r > 0) ? Hs + (r - 1) * MM : nullptr;   // H_{r, r-1} = R_{r-1} (upper)
    const double *hu = (r + 1 < steps) ? Hs + r * MM : nullptr; // H_{r, r+1} = R_r^T
    for (int idx = threadIdx.x; idx < M * TC; idx += blockDim.x) {
        const int i = idx / TC, cc = idx % TC, c = c0 + cc;
        if (c >= M) continue;
        double hv = 0.0;
        for (int k = 0; k < M; ++k) hv = fma(hd[i * M + k], s1[k * TC + cc], hv);
        if (hl)
            for (int k = i; k < M; ++k) hv = fma(hl[i * M + k], s0[k * TC + cc], hv);
        if (hu)
            for (int k = 0; k <= i; ++k) hv = fma(hu[k * M + i], s2[k * TC + cc], hv);
        const double av = s1[i * TC + cc] - g * hv;
        const int64_t o = r * MM + int64_t(i) * M + c;
        const double vn = beta * av - gamma * Vp[o];
        Vn[o] = vn;
        U[o] += dnext * vn;
    }
}

// ---------------------------------------------------------------- double-float recurrence
// The same recurrence with H and V held as unevaluated float pairs (hi + lo, about 48
// significant bits) on the FP32 pipe, which this part runs at 64 times its FP64 rate.  The
// products are compensated dot products (Ogita, Rump and Oishi's Dot2): each h v term is
// split exactly by an FMA (TwoProd), the running sum by Knuth's TwoSum, and the rounding
// errors are summed beside it; the result is exact to about 2^-48 relative, far below the
// 1e-14 the projected solve needs after thousands of terms.  U is accumulated in FP64.
struct dfl {
    float h, l;
};
__device__ __forceinline__ dfl dfl_fast(float s, float e) {   // |s| >= |e|
    const float h = s + e;
    return dfl{h, e - (h - s)};
}
// sum += a * b, exact products and sums tracked in (s, err)
__device__ __forceinline__ void dot2_step(float &s, float &err, dfl a, dfl b) {
    const float p = a.h * b.h;
    float pe = fmaf(a.h, b.h, -p);
    pe = fmaf(a.h, b.l, pe);
    pe = fmaf(a.l, b.h, pe);
    const float t = s + p;
    const float bb = t - s;
    err += ((s - (t - bb)) + (p - bb)) + pe;
    s = t;
}
__host__ __device__ __forceinline__ dfl dfl_from(double v) {
    const float h = float(v);
    return dfl{h, float(v - double(h))};
}
__device__ __forceinline__ double dfl_val(dfl a) { return double(a.h) + double(a.l); }

// H_d, H_s split into float pairs (once per projected solve)
__global__ void k_split_df(const double *__restrict__ H, dfl *__restrict__ out, int64_t count) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = dfl_from(H[i]);
}

__global__ void k_cheb_bt_seed_df(dfl *V0, double *U, int M, double d0, const Ctrl *ctrl) {
    const int i = threadIdx.x + blockIdx.x * blockDim.x;
    if (ctrl->steps > 0 && i < M) {
        V0[int64_t(i) * M + i] = dfl{1.f, 0.f};
        U[int64_t(i) * M + i] = d0;
    }
}

// V_{j+1} = beta (V_j - g H V_j) - gamma V_{j-1};  U += d_{j+1} V_{j+1}, in double-float
__global__ void __launch_bounds__(256)
k_cheb_bt_iter_df(const dfl *__restrict__ Hd, const dfl *__restrict__ Hs, const dfl *__restrict__ Vp,
                  const dfl *__restrict__ Vc, dfl *__restrict__ Vn, double *__restrict__ U, int M,
                  float beta, float gamma, double dnext, dfl g, const Ctrl *ctrl) {
    const int r = blockIdx.x;
    const int steps = ctrl->steps;
    if (r >= steps) return;
    const int c0 = blockIdx.y * TC;
    extern __shared__ __align__(16) unsigned char svraw[];   // [3][M][TC] pairs
    dfl *s0 = reinterpret_cast<dfl *>(svraw), *s1 = s0 + M * TC, *s2 = s0 + 2 * M * TC;
    const int64_t MM = int64_t(M) * M;
    for (int idx = threadIdx.x; idx < M * TC; idx += blockDim.x) {
        const int k = idx / TC, cc = idx % TC, c = c0 + cc;
        dfl a{0.f, 0.f}, b{0.f, 0.f}, d{0.f, 0.f};
        if (c < M) {
            if (r > 0) a = Vc[(r - 1) * MM + int64_t(k) * M + c];
            b = Vc[r * MM + int64_t(k) * M + c];
            if (r + 1 < steps) d = Vc[(r + 1) * MM + int64_t(k) * M + c];
        }
        s0[idx] = a; s1[idx] = b; s2[idx] = d;
    }
    __syncthreads();
    const dfl *hd = Hd + r * MM;
    const dfl *hl = (r > 0) ? Hs + (r - 1) * MM : nullptr;   // H_{r, r-1} = R_{r-1} (upper)
    const dfl *hu = (r + 1 < steps) ? Hs + r * MM : nullptr; // H_{r, r+1} = R_r^T
    for (int idx = threadIdx.x; idx < M * TC; idx += blockDim.x) {
        const int i = idx / TC, cc = idx % TC, c = c0 + cc;
        if (c >= M) continue;
        float s = 0.f, err = 0.f;
        for (int k = 0; k < M; ++k) dot2_step(s, err, hd[i * M + k], s1[k * TC + cc]);
        if (hl)
            for (int k = i; k < M; ++k) dot2_step(s, err, hl[i * M + k], s0[k * TC + cc]);
        if (hu)
            for (int k = 0; k <= i; ++k) dot2_step(s, err, hu[k * M + i], s2[k * TC + cc]);
        // av = V_j - g (H V_j): one more compensated step with the pair -g
        const dfl hv = dfl_fast(s, err);
        float s2v = s1[i * TC + cc].h, e2 = s1[i * TC + cc].l;
        dot2_step(s2v, e2, dfl{-g.h, -g.l}, hv);
        // vn = beta av - gamma V_{j-1} (beta in {1, 2}, gamma in {0, 1}: exact scalings)
        const int64_t o = r * MM + int64_t(i) * M + c;
        const dfl vp = Vp[o];
        float s3 = beta * s2v, e3 = beta * e2;
        dot2_step(s3, e3, dfl{-gamma, 0.f}, vp);
        const dfl vn = dfl_fast(s3, e3);
        Vn[o] = vn;
        U[o] += dnext * dfl_val(vn);
    }
}

// ---------------------------------------------------------------- block Cholesky (spline)
// One CTA; all scratch in global memory (L1/L2 resident for the sizes used).
__device__ void chol_lower_inplace(double *A, int M) {
    // A = L L^T, lower L overwrites A (upper part left as is); the trailing update runs rows
    // by warp and columns by lane (no index division, no idle half)
    __shared__ double piv, rpiv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < M; ++j) {
        if (threadIdx.x == 0) {
            double d = A[j * M + j];
            piv = sqrt(fmax(d, 1e-300));
            rpiv = 1.0 / piv;
            A[j * M + j] = piv;
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < M; i += blockDim.x) A[i * M + j] *= rpiv;
        __syncthreads();
        for (int a = j + 1 + warp; a < M; a += nw) {
            const double laj = A[a * M + j];
            for (int b = j + 1 + lane; b <= a; b += 32) A[a * M + b] -= laj * A[b * M + j];
        }
        __syncthreads();
    }
}

// Block Cholesky factorisation eps I + H = L L^T of the block tridiagonal Lanczos matrix (L
// block lower bidiagonal: lower triangular diagonal blocks Ld_r, sub-diagonal blocks Ls_r),
// block by block, three launches per block (FP64 runs at a small fraction of the FP32 rate
// on this part, so the dense parts are spread over as many SMs as there are rows):
//   k_bt_dupdate  D_r = eps I + H_rr - Ls_{r-1} Ls_{r-1}^T (lower triangle), one CTA per row
//   k_bt_dchol    D_r = Ld_r Ld_r^T in place, one CTA
//   k_bt_lsolve   Ls_r = H_{r+1,r} Ld_r^{-T}, one warp per row
// Each launch does nothing when its block lies past ctrl->steps.
__global__ void __launch_bounds__(128)
k_bt_dupdate(const double *__restrict__ Hd, const double *__restrict__ Ls, int M, double eps, int r,
             double *__restrict__ Ld, const Ctrl *ctrl) {
    if (r >= ctrl->steps) return;
    const int i = blockIdx.x;
    const int64_t MM = int64_t(M) * M;
    const double *P = r > 0 ? Ls + (r - 1) * MM : nullptr;
    double *D = Ld + r * MM;
    for (int j = threadIdx.x; j <= i; j += blockDim.x) {
        double v = Hd[r * MM + int64_t(i) * M + j] + (i == j ? eps : 0.0);
        if (P)
            for (int k = 0; k < M; ++k) v = fma(-P[int64_t(i) * M + k], P[int64_t(j) * M + k], v);
        D[int64_t(i) * M + j] = v;
    }
}

__global__ void __launch_bounds__(1024) k_bt_dchol(double *Ld, int M, int r, const Ctrl *ctrl) {
    if (r >= ctrl->steps) return;
    chol_lower_inplace(Ld + r * int64_t(M) * M, M);
}

// Row i of Ls_r solves Ld_r x = (row i of H_{r+1,r})^T by column-oriented forward substitution
// with x in registers (lane l: entries l, l + 32, l + 64, l + 96; M <= 128): x_j = y_j / d_jj,
// then y_k -= d_kj x_j for the rows k below, one shuffle per row.
__global__ void __launch_bounds__(32)
k_bt_lsolve(const double *__restrict__ Hs, const double *__restrict__ Ld, int M, int r,
            double *__restrict__ Ls, const Ctrl *ctrl) {
    if (r + 1 >= ctrl->steps) return;
    const int i = blockIdx.x, lane = threadIdx.x;
    const int64_t MM = int64_t(M) * M;
    const double *D = Ld + r * MM;
    const double *h = Hs + r * MM + int64_t(i) * M;
    double y[4], rd[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = lane + 32 * q;
        y[q] = j < M ? h[j] : 0.0;
        rd[q] = 1.0 / (j < M ? D[int64_t(j) * M + j] : 1.0);
    }
#pragma unroll
    for (int jq = 0; jq < 4; ++jq)
        for (int jl = 0; jl < 32; ++jl) {
            const int j = 32 * jq + jl;
            if (j >= M) break;
            const double xj = __shfl_sync(0xffffffffu, y[jq], jl) * __shfl_sync(0xffffffffu, rd[jq], jl);
            if (lane == jl) y[jq] = xj;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = lane + 32 * q;
                if (k > j && k < M) y[q] = fma(-D[int64_t(k) * M + j], xj, y[q]);
            }
        }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = lane + 32 * q;
        if (j < M) Ls[r * MM + int64_t(i) * M + j] = y[q];
    }
}

// s_int times U <- (eps I + H)^{-1} U with the factors Ld, Ls (k_bt_dupdate / dchol / lsolve), by forward and
// backward block substitution; U starts as F_1 = [I; 0; ...] unless rhs_in_u (U already holds
// the right-hand side, steps blocks).  The right-hand-side columns are independent: one warp
// per column, BTS_COLS columns per CTA, the CTAs side by side (FP64 runs at a small fraction
// of the FP32 rate on this part, so the columns are spread over as many SMs as there are).  A
// warp keeps its column of the current block in registers (lane l: rows l, l + 32, l + 64,
// l + 96; M <= 128), takes the coupling term Ls y from the previous block's column (broadcast
// by shuffles) and solves the triangular system column-oriented: y_i /= d_ii, then
// y_k -= d_ki y_i for the rows k below (k above in the backward solve with D^T), one shuffle
// per row.  No block barrier is used.  Yw holds the forward solutions Y_r for the backward
// pass.
constexpr int BTS_COLS = 1;
constexpr int BTS_R = 4;   // rows per lane
__global__ void __launch_bounds__(32 * BTS_COLS)
k_bt_spline_subst(const double *__restrict__ Ld, const double *__restrict__ Ls, int M, int s_int,
                  double *__restrict__ Yw, double *__restrict__ U, const Ctrl *ctrl, int rhs_in_u) {
    const int steps = ctrl->steps;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * BTS_COLS + (threadIdx.x >> 5);
    if (c >= M) return;   // whole warps: nothing below synchronises the block
    const int64_t MM = int64_t(M) * M;
    double y[BTS_R], yp[BTS_R], rd[BTS_R];
    for (int rep = 0; rep < s_int; ++rep) {
        // forward: Y_r = D_r^{-1} (U_r - Ls_{r-1} Y_{r-1})
        for (int r = 0; r < steps; ++r) {
            const double *D = Ld + r * MM;
#pragma unroll
            for (int q = 0; q < BTS_R; ++q) {
                const int i = lane + 32 * q;
                double v = 0.0, d = 1.0;
                if (i < M) {
                    v = (rep == 0 && !rhs_in_u) ? ((r == 0 && i == c) ? 1.0 : 0.0) : U[r * MM + int64_t(i) * M + c];
                    d = D[int64_t(i) * M + i];
                }
                y[q] = v;
                rd[q] = 1.0 / d;
            }
            if (r > 0) {
                const double *P = Ls + (r - 1) * MM;
#pragma unroll
                for (int kq = 0; kq < BTS_R; ++kq)
                    for (int kl = 0; kl < 32; ++kl) {
                        const int k = 32 * kq + kl;
                        if (k >= M) break;
                        const double ypk = __shfl_sync(0xffffffffu, yp[kq], kl);
#pragma unroll
                        for (int q = 0; q < BTS_R; ++q) {
                            const int i = lane + 32 * q;
                            if (i < M) y[q] = fma(-P[int64_t(i) * M + k], ypk, y[q]);
                        }
                    }
            }
#pragma unroll
            for (int iq = 0; iq < BTS_R; ++iq)
                for (int il = 0; il < 32; ++il) {
                    const int i = 32 * iq + il;
                    if (i >= M) break;
                    const double yi = __shfl_sync(0xffffffffu, y[iq], il) * __shfl_sync(0xffffffffu, rd[iq], il);
                    if (lane == il) y[iq] = yi;
#pragma unroll
                    for (int q = 0; q < BTS_R; ++q) {
                        const int k = lane + 32 * q;
                        if (k > i && k < M) y[q] = fma(-D[int64_t(k) * M + i], yi, y[q]);
                    }
                }
#pragma unroll
            for (int q = 0; q < BTS_R; ++q) {
                const int i = lane + 32 * q;
                if (i < M) Yw[r * MM + int64_t(i) * M + c] = y[q];
                yp[q] = y[q];
            }
        }
        // backward: U_r = D_r^{-T} (Y_r - Ls_r^T U_{r+1})
        for (int r = steps - 1; r >= 0; --r) {
            const double *D = Ld + r * MM;
#pragma unroll
            for (int q = 0; q < BTS_R; ++q) {
                const int i = lane + 32 * q;
                y[q] = i < M ? Yw[r * MM + int64_t(i) * M + c] : 0.0;
                rd[q] = 1.0 / (i < M ? D[int64_t(i) * M + i] : 1.0);
            }
            if (r + 1 < steps) {
                const double *P = Ls + r * MM;
#pragma unroll
                for (int kq = 0; kq < BTS_R; ++kq)
                    for (int kl = 0; kl < 32; ++kl) {
                        const int k = 32 * kq + kl;
                        if (k >= M) break;
                        const double unk = __shfl_sync(0xffffffffu, yp[kq], kl);
#pragma unroll
                        for (int q = 0; q < BTS_R; ++q) {
                            const int i = lane + 32 * q;
                            if (i < M) y[q] = fma(-P[int64_t(k) * M + i], unk, y[q]);
                        }
                    }
            }
#pragma unroll
            for (int iq = BTS_R - 1; iq >= 0; --iq)
                for (int il = 31; il >= 0; --il) {
                    const int i = 32 * iq + il;
                    if (i >= M) continue;
                    const double ui = __shfl_sync(0xffffffffu, y[iq], il) * __shfl_sync(0xffffffffu, rd[iq], il);
                    if (lane == il) y[iq] = ui;
#pragma unroll
                    for (int q = 0; q < BTS_R; ++q) {
                        const int k = lane + 32 * q;
                        if (k < i) y[q] = fma(-D[int64_t(i) * M + k], ui, y[q]);
                    }
                }
#pragma unroll
            for (int q = 0; q < BTS_R; ++q) {
                const int i = lane + 32 * q;
                if (i < M) U[r * MM + int64_t(i) * M + c] = y[q];
                yp[q] = y[q];
            }
        }
    }
}

// ---------------------------------------------------------------- quadrature nodes (spline)
// One CTA per quadrature node: Y = (sigma I + H)^{-1} F_1 through the block Cholesky
// factorisation sigma I + H = L L^T (L block lower bidiagonal: diagonal blocks Ld_r lower
// triangular, sub-diagonal blocks Ls_r = L_{r+1,r}), forward and backward block substitution.
// The triangular solves give each thread one row (Ls) or one right-hand-side column (Y), so
// they need no barrier inside a block.  Per-node scratch (bt_quad_node_doubles): Ld, Ls, Y
// (mcap blocks of M x M each) and the reciprocal diagonals of the Ld blocks (mcap x M).
constexpr int QN_THREADS = 128;

__global__ void __launch_bounds__(QN_THREADS)
k_bt_shift_solve(const double *__restrict__ Hd, const double *__restrict__ Hs, int M, int mcap,
                 QuadRule q, int node0, double *scratch, const Ctrl *ctrl) {
    const int node = node0 + int(blockIdx.x);
    if (node >= q.n) return;
    const int steps = ctrl->steps;
    const double sigma = q.shift[node];
    const int64_t MM = int64_t(M) * M;
    double *Ld = scratch + int64_t(blockIdx.x) * int64_t(bt_quad_node_doubles(M, mcap));
    double *Ls = Ld + int64_t(mcap) * MM;
    double *Y = Ls + int64_t(mcap) * MM;
    double *rd = Y + int64_t(mcap) * MM;
    const int tid = threadIdx.x;
    for (int r = 0; r < steps; ++r) {
        // D_r = sigma I + H_rr - Ls_{r-1} Ls_{r-1}^T (lower triangle), then D_r = Ld_r Ld_r^T
        double *D = Ld + r * MM;
        const double *P = r > 0 ? Ls + (r - 1) * MM : nullptr;
        for (int idx = tid; idx < M * M; idx += blockDim.x) {
            const int i = idx / M, j = idx % M;
            double v = 0.0;
            if (j <= i) {
                v = Hd[r * MM + idx] + (i == j ? sigma : 0.0);
                if (P)
                    for (int k = 0; k < M; ++k) v = fma(-P[i * M + k], P[j * M + k], v);
            }
            D[idx] = v;
        }
        __syncthreads();
        chol_lower_inplace(D, M);
        for (int i = tid; i < M; i += blockDim.x) rd[r * M + i] = 1.0 / D[i * M + i];
        __syncthreads();
        if (r + 1 < steps) {
            // Ls_r = H_{r+1,r} D_r^{-T}: row i solves D_r x = (row i of H_{r+1,r})^T
            const double *Hsub = Hs + r * MM;
            double *Pn = Ls + r * MM;
            for (int i = tid; i < M; i += blockDim.x)
                for (int j = 0; j < M; ++j) {
                    double v = Hsub[i * M + j];
                    for (int k = 0; k < j; ++k) v = fma(-D[j * M + k], Pn[i * M + k], v);
                    Pn[i * M + j] = v * rd[r * M + j];
                }
            __syncthreads();
        }
    }
    // forward: Y_0 = D_0^{-1} I, Y_r = D_r^{-1} (-Ls_{r-1} Y_{r-1}); one column per thread
    for (int r = 0; r < steps; ++r) {
        const double *D = Ld + r * MM;
        const double *P = r > 0 ? Ls + (r - 1) * MM : nullptr;
        const double *Yp = r > 0 ? Y + (r - 1) * MM : nullptr;
        double *Yr = Y + r * MM;
        for (int c = tid; c < M; c += blockDim.x)
            for (int i = 0; i < M; ++i) {
                double v = (r == 0 && i == c) ? 1.0 : 0.0;
                if (P)
                    for (int k = 0; k < M; ++k) v = fma(-P[i * M + k], Yp[k * M + c], v);
                for (int k = 0; k < i; ++k) v = fma(-D[i * M + k], Yr[k * M + c], v);
                Yr[i * M + c] = v * rd[r * M + i];
            }
        __syncthreads();
    }
    // backward: U_r = D_r^{-T} (Y_r - Ls_r^T U_{r+1}), in place in Y
    for (int r = steps - 1; r >= 0; --r) {
        const double *D = Ld + r * MM;
        const double *P = r + 1 < steps ? Ls + r * MM : nullptr;
        const double *Un = r + 1 < steps ? Y + (r + 1) * MM : nullptr;
        double *Yr = Y + r * MM;
        for (int c = tid; c < M; c += blockDim.x)
            for (int i = M - 1; i >= 0; --i) {
                double v = Yr[i * M + c];
                if (P)
                    for (int k = 0; k < M; ++k) v = fma(-P[k * M + i], Un[k * M + c], v);
                for (int k = i + 1; k < M; ++k) v = fma(-D[k * M + i], Yr[k * M + c], v);
                Yr[i * M + c] = v * rd[r * M + i];
            }
        __syncthreads();
    }
}

// U += sum_{j < nb} W_{node0+j} Y_j over the steps blocks, in a fixed order (deterministic).
__global__ void __launch_bounds__(256)
k_quad_accumulate(const double *__restrict__ scratch, int M, int mcap, int nb, QuadRule q, int node0,
                  double *U, const Ctrl *ctrl) {
    const int64_t cnt = int64_t(ctrl->steps) * M * M;
    const int64_t per = int64_t(bt_quad_node_doubles(M, mcap));
    const int64_t yoff = 2 * int64_t(mcap) * M * M;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < cnt;
         idx += int64_t(gridDim.x) * blockDim.x) {
        double acc = U[idx];
        for (int j = 0; j < nb; ++j) acc = fma(q.weight[node0 + j], scratch[j * per + yoff + idx], acc);
        U[idx] = acc;
    }
}

}  // namespace

int launch_cheb_bt(const double *Hd, const double *Hs, int M, int m, double lam,
                   const std::vector<double> &d, double *V0, double *V1, double *V2, double *U,
                   const Ctrl *ctrl, cudaStream_t s, double *Hdf) {
    const size_t bytes = sizeof(double) * size_t(m) * M * M;
    prof_begin(KernelClass::PROJECTED, s);
    if (Hdf) {
        // double-float recurrence: H split once, V_j as float pairs in the V buffers
        const int64_t cnt = int64_t(m) * M * M;
        dfl *hd = reinterpret_cast<dfl *>(Hdf), *hs = hd + cnt;
        const int sg = int(std::min<int64_t>((cnt + 255) / 256, 8 * int64_t(num_sms())));
        k_split_df<<<sg, 256, 0, s>>>(Hd, hd, cnt);
        k_split_df<<<sg, 256, 0, s>>>(Hs, hs, cnt);
        KB_CUDA_TRY(cudaMemsetAsync(V0, 0, bytes, s));
        KB_CUDA_TRY(cudaMemsetAsync(V1, 0, bytes, s));
        KB_CUDA_TRY(cudaMemsetAsync(V2, 0, bytes, s));
        zero_if_active(U, int64_t(m) * M * M, ctrl, s);
        dfl *pp = reinterpret_cast<dfl *>(V2), *pc = reinterpret_cast<dfl *>(V0), *pn = reinterpret_cast<dfl *>(V1);
        k_cheb_bt_seed_df<<<(M + 127) / 128, 128, 0, s>>>(pc, U, M, d[0], ctrl);
        const size_t smem = sizeof(dfl) * 3 * M * TC;
        const dfl g = dfl_from(2.0 / lam);
        for (size_t j = 0; j + 1 < d.size(); ++j) {
            const int nrb = std::min<int>(int(j) + 2, m);
            dim3 grid(nrb, (M + TC - 1) / TC);
            const float beta = j == 0 ? 1.f : 2.f, gamma = j == 0 ? 0.f : 1.f;
            k_cheb_bt_iter_df<<<grid, 256, smem, s>>>(hd, hs, pp, pc, pn, U, M, beta, gamma, d[j + 1], g, ctrl);
            dfl *t = pp; pp = pc; pc = pn; pn = t;
        }
        KB_CUDA_TRY(cudaGetLastError());
        prof_end(KernelClass::PROJECTED, s, 0, 0, int(d.size()) + 3);
        return 0;
    }
    KB_CUDA_TRY(cudaMemsetAsync(V0, 0, bytes, s));
    KB_CUDA_TRY(cudaMemsetAsync(V1, 0, bytes, s));
    KB_CUDA_TRY(cudaMemsetAsync(V2, 0, bytes, s));
    zero_if_active(U, int64_t(m) * M * M, ctrl, s);
    k_cheb_bt_seed<<<(M + 127) / 128, 128, 0, s>>>(V0, U, M, d[0], ctrl);
    const size_t smem = sizeof(double) * 3 * M * TC;
    // function-local static: initialised once, thread-safe (several serving workers)
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_cheb_bt_iter, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(double) * 3 * 128 * TC));
    (void)attr;
    double *pp = V2, *pc = V0, *pn = V1;
    const double g = 2.0 / lam;
    for (size_t j = 0; j + 1 < d.size(); ++j) {
        const int nrb = std::min<int>(int(j) + 2, m);
        dim3 grid(nrb, (M + TC - 1) / TC);
        const double beta = j == 0 ? 1.0 : 2.0, gamma = j == 0 ? 0.0 : 1.0;
        k_cheb_bt_iter<<<grid, 256, smem, s>>>(Hd, Hs, pp, pc, pn, U, M, beta, gamma, d[j + 1], g, ctrl);
        double *t = pp; pp = pc; pc = pn; pn = t;
    }
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::PROJECTED, s, 0, 0, int(d.size()));
    return 0;
}

// The block factorisation, launched block by block up to kmax; returns the launch count.
static int bt_factor(const double *Hd, const double *Hs, int M, int kmax, double eps, double *Ld,
                     double *Ls, const Ctrl *ctrl, cudaStream_t s) {
    for (int r = 0; r < kmax; ++r) {
        k_bt_dupdate<<<M, 128, 0, s>>>(Hd, Ls, M, eps, r, Ld, ctrl);
        k_bt_dchol<<<1, 1024, 0, s>>>(Ld, M, r, ctrl);
        if (r + 1 < kmax) k_bt_lsolve<<<M, 32, 0, s>>>(Hs, Ld, M, r, Ls, ctrl);
    }
    return 3 * kmax - 1;
}

int launch_bt_spline(const double *Hd, const double *Hs, int M, int m, double eps, int s_int,
                     double *Ld, double *Ls, double *Yw, double *U, const Ctrl *ctrl,
                     cudaStream_t s, const QuadRule *q, double *qscr, int qbatch, int kmax) {
    if (kmax <= 0 || kmax > m) kmax = m;
    prof_begin(KernelClass::PROJECTED, s);
    int launches = 1;   // zero_if_active
    if (q && q->n > 0) {
        if (!qscr || qbatch < 1) return fail(KB_ERR_ARG, "spline quadrature without scratch");
        zero_if_active(U, int64_t(m) * M * M, ctrl, s);
        const int acc_grid = int(std::min<int64_t>((int64_t(m) * M * M + 255) / 256, 4 * int64_t(num_sms())));
        for (int j0 = 0; j0 < q->n; j0 += qbatch) {
            const int nb = std::min(qbatch, q->n - j0);
            k_bt_shift_solve<<<nb, QN_THREADS, 0, s>>>(Hd, Hs, M, m, *q, j0, qscr, ctrl);
            k_quad_accumulate<<<std::max(acc_grid, 1), 256, 0, s>>>(qscr, M, m, nb, *q, j0, U, ctrl);
            launches += 2;
        }
        if (s_int > 0) {
            launches += bt_factor(Hd, Hs, M, kmax, eps, Ld, Ls, ctrl, s) + 1;
            k_bt_spline_subst<<<(M + BTS_COLS - 1) / BTS_COLS, 32 * BTS_COLS, 0, s>>>(Ld, Ls, M, s_int, Yw, U, ctrl, 1);
        }
    } else {
        // (blocks past the steps stay zero: the bound check reads all m of them)
        zero_if_active(U, int64_t(m) * M * M, ctrl, s);
        launches += bt_factor(Hd, Hs, M, kmax, eps, Ld, Ls, ctrl, s);
        k_bt_spline_subst<<<(M + BTS_COLS - 1) / BTS_COLS, 32 * BTS_COLS, 0, s>>>(Ld, Ls, M, s_int, Yw, U, ctrl, 0);
        ++launches;
    }
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::PROJECTED, s, 0, 0, launches);
    return 0;
}

}  // namespace kb
