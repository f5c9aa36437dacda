// Small dense FP64 kernels and element-wise kernels of the Krylov drivers.
//
//  * k_hkk          symmetrised diagonal block H_kk (Algorithm 1, line 4).
//  * k_chol         reduced QR of the new block by CholeskyQR, FP64 Cholesky factor and its
//                   inverse (Algorithm 1, line 6); the second pass forms H_{k+1,k} = R2 R1
//                   and the transposed block used by the next three-term step (line 7,
//                   reading A1).  Invariant subspaces stop the process, rank-deficient
//                   blocks report a breakdown (reading A6).
//  * k_lanczos_*    scalar recurrences of the global (Algorithm 2) and sequential
//                   (Section 3.3) Lanczos methods: h_kk, h_{k+1,k}, 1/h.
//  * k_tridiag_phi  u = phi(H_m) f_1 for the tridiagonal Lanczos matrices (Algorithm 2,
//                   line 8; Section 3.3 with phi applied, reading A2).
//  * element-wise   unit blocks E_W, node markers, column norms, scaled copies, the
//                   diagonal assembly sum_k u_k Q_k, NaN fill on breakdown.
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

// ---------------------------------------------------------------- control / init
__global__ void k_ctrl_init(Ctrl *c, int steps) {
    c->status = KB_OK;
    c->stop = 0;
    c->steps = steps;
    c->breakdown_step = -1;
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
        out[i] = T(scale * double(in[i]));
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
__global__ void k_hkk(const double *G, int M, int W, double *Hd, T *C, const Ctrl *ctrl) {
    if (ctrl->stop) return;
    for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
        const int i = idx / W, j = idx % W;
        double v = 0.0;
        if (i < M && j < M) v = 0.5 * (G[i * W + j] + G[j * W + i]);
        // recorded exactly as the update subtracts it (rounded to the basis precision)
        const T vt = T(v);
        if (i < M && j < M) Hd[i * M + j] = double(vt);
        C[idx] = vt;
    }
}

// In-place inverse of an upper triangular M x M matrix in shared memory (ld lda), column
// by column: with the leading j x j block already inverted, column j of the inverse is
// -(1/a_jj) X_{0:j,0:j} a_{0:j,j}.  Each row's dot product is split over TPR consecutive
// lanes (TPR = 1, 2, 4 or 8) and combined with shuffles.  t: shared scratch of M doubles.
__device__ void tri_inv_upper_inplace(double *A, int lda, int M, double *t) {
    int TPR = 1;
    while (TPR < 8 && TPR * 2 * M <= int(blockDim.x)) TPR *= 2;
    const int sub = threadIdx.x % TPR;
    const int row0 = threadIdx.x / TPR;
    const int rstride = blockDim.x / TPR;
    for (int j = 0; j < M; ++j) {
        for (int i = threadIdx.x; i < j; i += blockDim.x) t[i] = A[i * lda + j];
        __syncthreads();
        const double ajj = 1.0 / A[j * lda + j];
        // rows i < j, all TPR lanes of a row iterate together (uniform loop bound per warp)
        for (int ib = 0; ib < j; ib += rstride) {
            const int i = ib + row0;
            double acc = 0.0;
            if (i < j)
                for (int k = i + sub; k < j; k += TPR) acc = fma(A[i * lda + k], t[k], acc);
            for (int off = 1; off < TPR; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (i < j && sub == 0) A[i * lda + j] = -ajj * acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) A[j * lda + j] = ajj;
        __syncthreads();
    }
}

// Cholesky G = R^T R (upper R) of the leading M x M block in shared memory, then R^{-1}.
template <typename T>
__global__ void __launch_bounds__(256) k_chol(const double *G, int M, int W, int pass, int step,
                                              double inv_thresh2, double piv_rel2, double *R1,
                                              T *Rinv, double *Hs, T *Bout, Ctrl *ctrl) {
    if (ctrl->stop) return;
    extern __shared__ double A[];   // [M][M+1], then t[M]
    __shared__ int bad;
    __shared__ double maxdiag;
    const int lda = M + 1;
    double *t = A + M * lda;
    for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
        const int i = idx / M, j = idx % M;
        A[i * lda + j] = G[i * W + j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, mx = 0.0;
        for (int i = 0; i < M; ++i) { tr += A[i * lda + i]; mx = fmax(mx, A[i * lda + i]); }
        maxdiag = mx;
        bad = 0;
        if (pass == 1 && !(tr > inv_thresh2)) {
            // X vanished: the block Krylov space is invariant; keep the blocks so far
            ctrl->stop = 1;
            ctrl->steps = step;
            bad = 2;
        }
    }
    __syncthreads();
    if (bad) return;
    for (int j = 0; j < M; ++j) {
        if (threadIdx.x == 0) {
            const double d = A[j * lda + j];
            if (!(d > piv_rel2 * maxdiag)) {
                bad = 1;
                ctrl->status = KB_ERR_BREAKDOWN;
                ctrl->stop = 1;
                ctrl->steps = step;
                ctrl->breakdown_step = step;
            } else {
                const double r = sqrt(d);
                A[j * lda + j] = r;
                t[0] = 1.0 / r;
            }
        }
        __syncthreads();
        if (bad) return;
        const double rinv = t[0];
        for (int c = j + 1 + threadIdx.x; c < M; c += blockDim.x) A[j * lda + c] *= rinv;
        __syncthreads();
        const int L = M - j - 1;
        const int npairs = L * (L + 1) / 2;
        for (int idx = threadIdx.x; idx < npairs; idx += blockDim.x) {
            // idx -> (a, b), a <= b, in the trailing upper triangle (FP32 root estimate,
            // corrected exactly in integers)
            int a = int((sqrtf(8.f * float(idx) + 1.f) - 1.f) * 0.5f);
            while ((a + 1) * (a + 2) / 2 <= idx) ++a;
            while (a * (a + 1) / 2 > idx) --a;
            const int b = idx - a * (a + 1) / 2;   // 0 <= b <= a
            const int ra = j + 1 + b, rb = j + 1 + a;   // ra <= rb
            A[ra * lda + rb] -= A[j * lda + ra] * A[j * lda + rb];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
        const int i = idx / M, j = idx % M;
        if (j < i) A[i * lda + j] = 0.0;
    }
    __syncthreads();
    // R^{-1} (upper triangular), in place
    tri_inv_upper_inplace(A, lda, M, t);
    for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
        const int i = idx / W, j = idx % W;
        const T v = (i < M && j < M && j >= i) ? T(A[i * lda + j]) : T(0);
        Rinv[idx] = v;
        if (i < M && j < M) A[i * lda + j] = double(v);
    }
    __syncthreads();
    // The row-block kernels apply the inverse rounded to the basis precision.  Record the
    // factor actually applied, the FP64 inverse of the rounded inverse, so that
    // X = Q_{k+1} H_{k+1,k} holds for the stored blocks up to the rounding of Q.
    tri_inv_upper_inplace(A, lda, M, t);
    if (pass == 1) {
        for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
            const int i = idx / M, j = idx % M;
            R1[idx] = (j >= i) ? A[i * lda + j] : 0.0;
        }
    } else {
        // H_{k+1,k} = R2 R1 (upper triangular); B = H^T for the next three-term step.  H is
        // recorded rounded to the basis precision, i.e. exactly as the next step subtracts it.
        for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
            const int i = idx / W, j = idx % W;
            double h = 0.0;
            if (i < M && j < M && j >= i) {
                for (int k = i; k <= j; ++k) h = fma(A[i * lda + k], __ldg(R1 + k * M + j), h);
            }
            const T ht = T(h);
            if (i < M && j < M) Hs[i * M + j] = double(ht);
            Bout[j * W + i] = ht;
        }
    }
}

// ---------------------------------------------------------------- gbl / sbl scalars
// Reduce [nparts][W] partials per column (fixed order) into s[W].
__device__ void reduce_cols(const double *parts, int nparts, int W, double *s) {
    __shared__ double tmp[8][128];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < W; c0 += 32) {
        const int c = c0 + lane;
        double acc = 0.0;
        if (c < W)
            for (int p = warp; p < nparts; p += 8) acc += parts[int64_t(p) * W + c];
        if (c < W) tmp[warp][c] = acc;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += tmp[w][c];
        s[c] = t;
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

// alpha_k = <Q_k, X> (gbl: Frobenius, sbl: per column) from SpMM dot partials of P_k . X
__global__ void k_lanczos_alpha(const double *parts, int nparts, int W, int M, int gbl, int k,
                                const double *sigma, double *alpha, double *a_upd, const Ctrl *ctrl) {
    if (ctrl->stop) return;
    __shared__ double s[128];
    reduce_cols(parts, nparts, W, s);
    const double *sg = sigma + int64_t(k) * W;
    if (gbl) {
        __shared__ double tot;
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int c = 0; c < M; ++c) t += s[c];
            tot = sg[0] * t;
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
    reduce_cols(parts, nparts, W, s);
    const double *sk = sigma + int64_t(k) * W;
    double *sn = sigma + int64_t(k + 1) * W;
    double *bn = beta + int64_t(k + 1) * W;
    if (gbl) {
        __shared__ double b;
        __shared__ int stop;
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int c = 0; c < M; ++c) t += s[c];
            b = sqrt(t);
            stop = !(b > thresh);
            if (stop) { ctrl->stop = 1; ctrl->steps = k + 1; }
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
//   spline: s_int solves with the SPD tridiagonal eps I + T (Thomas algorithm)
__global__ void k_tridiag_phi(int W, int M, int m, int gbl, const double *alpha,
                              const double *beta, const double *sigma, int phi_kind,
                              double eps, int s_int, double lam, ChebCoef cc, double *omega,
                              double *work, const Ctrl *ctrl) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncol = gbl ? 1 : M;
    if (c >= W) return;
    const int steps = gbl ? ctrl->steps : m;
    if (c >= ncol) {
        if (!gbl)
            for (int k = 0; k < m; ++k) omega[int64_t(k) * W + c] = 0.0;
        return;
    }
    // per-thread work vectors in global scratch: 4 vectors of length m
    double *v0 = work + int64_t(c) * 4 * m;
    double *v1 = v0 + m, *v2 = v1 + m, *u = v2 + m;
    auto a_of = [&](int k) { return alpha[int64_t(k) * W + c]; };
    auto b_of = [&](int k) { return beta[int64_t(k) * W + c]; };   // couples k-1 and k
    const int s = steps;
    for (int k = 0; k < s; ++k) { v0[k] = 0.0; v1[k] = 0.0; v2[k] = 0.0; u[k] = 0.0; }
    if (phi_kind == KB_PHI_EXP) {
        // v0 = e_1, v1 = A e_1, v_{j+1} = 2 A v_j - v_{j-1}, A = I - (2/lam) T
        const double g = 2.0 / lam;
        v0[0] = 1.0;
        u[0] = cc.d[0];
        double *pp = v0, *pc = v1, *pn = v2;
        // pc = A pp
        for (int k = 0; k < s; ++k) {
            double tv = a_of(k) * pp[k];
            if (k > 0) tv += b_of(k) * pp[k - 1];
            if (k + 1 < s) tv += b_of(k + 1) * pp[k + 1];
            pc[k] = pp[k] - g * tv;
            u[k] += cc.d[1] * pc[k];
        }
        for (int j = 2; j < cc.n; ++j) {
            for (int k = 0; k < s; ++k) {
                double tv = a_of(k) * pc[k];
                if (k > 0) tv += b_of(k) * pc[k - 1];
                if (k + 1 < s) tv += b_of(k + 1) * pc[k + 1];
                pn[k] = 2.0 * (pc[k] - g * tv) - pp[k];
                u[k] += cc.d[j] * pn[k];
            }
            double *t = pp; pp = pc; pc = pn; pn = t;
        }
    } else {
        // Thomas algorithm for (eps I + T) x = rhs, repeated s_int times from rhs = e_1
        u[0] = 1.0;
        for (int rep = 0; rep < s_int; ++rep) {
            // forward elimination: v0 = modified super-diagonal, v1 = modified rhs
            double den = eps + a_of(0);
            v0[0] = (s > 1) ? b_of(1) / den : 0.0;
            v1[0] = u[0] / den;
            for (int k = 1; k < s; ++k) {
                den = eps + a_of(k) - b_of(k) * v0[k - 1];
                v0[k] = (k + 1 < s) ? b_of(k + 1) / den : 0.0;
                v1[k] = (u[k] - b_of(k) * v1[k - 1]) / den;
            }
            u[s - 1] = v1[s - 1];
            for (int k = s - 2; k >= 0; --k) u[k] = v1[k] - v0[k] * u[k + 1];
        }
    }
    // E_W = P_1 and Q_1 = sigma_1 P_1, so Y = (1/sigma_1) [Q_1..Q_m] phi(T) e_1
    // (sqrt(N) of Algorithm 2, line 8, for the global method)
    const double scale = 1.0 / sigma[c];
    for (int k = 0; k < m; ++k) {
        double om = 0.0;
        if (k < s) om = scale * u[k] * sigma[int64_t(k) * W + c];
        if (gbl) {
            for (int cc2 = 0; cc2 < W; ++cc2)
                omega[int64_t(k) * W + cc2] = cc2 < M ? om : 0.0;
        } else {
            omega[int64_t(k) * W + c] = om;
        }
    }
}

// X[:, c] -= a[c] * P[:, c]; partial column sums of X^2 per CTA
template <typename T, int W>
__global__ void __launch_bounds__(256) k_axpy_colnorm(T *X, const T *P, const double *a, int64_t n,
                                                       double *parts, const Ctrl *ctrl) {
    if (ctrl->stop) return;
    constexpr int CG = W / 4;
    constexpr int RPP = 256 / CG;   // rows per pass
    __shared__ double s[RPP][W];
    const int cg = threadIdx.x % CG, rr = threadIdx.x / CG;
    const int c4 = cg * 4;
    T ah[4], al[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        ah[q] = T(a[c4 + q]);
        al[q] = T(a[c4 + q] - double(ah[q]));
    }
    T acc[4] = {0, 0, 0, 0};
    // two rows per iteration, 16-byte vector accesses: four loads in flight per thread
    const int64_t stride = int64_t(gridDim.x) * RPP;
    for (int64_t row = int64_t(blockIdx.x) * RPP + rr; row < n; row += 2 * stride) {
        const int64_t row2 = row + stride;
        T xv[2][4], pv[2][4];
        ldv4(X + row * W + c4, xv[0]);
        ldv4(P + row * W + c4, pv[0]);
        if (row2 < n) {
            ldv4(X + row2 * W + c4, xv[1]);
            ldv4(P + row2 * W + c4, pv[1]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && row2 >= n) break;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                xv[h][q] = xv[h][q] - fma(ah[q], pv[h][q], al[q] * pv[h][q]);
                acc[q] = fma(xv[h][q], xv[h][q], acc[q]);
            }
            stv4(X + (h ? row2 : row) * W + c4, xv[h]);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) s[rr][c4 + q] = acc[q];
    __syncthreads();
    for (int c = threadIdx.x; c < W; c += 256) {
        double t = 0.0;
        for (int r = 0; r < RPP; ++r) t += s[r][c];
        parts[int64_t(blockIdx.x) * W + c] = t;
    }
}

// Y[i, c] = sum_k omega_k[c] P_k[i, c]  (global / sequential Lanczos assembly)
template <typename T, int W>
__global__ void __launch_bounds__(256) k_assemble_diag(const T *basis, int64_t stride, int nblk,
                                                        const double *omega, int64_t n, float *Y,
                                                        int64_t ldy, int mo) {
    constexpr int CG = W / 4;
    constexpr int RPP = 256 / CG;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *som = reinterpret_cast<T *>(sm_raw);     // [nblk][W]
    for (int i = threadIdx.x; i < nblk * W; i += blockDim.x) som[i] = T(omega[i]);
    __syncthreads();
    const int cg = threadIdx.x % CG, rr = threadIdx.x / CG;
    const int c4 = cg * 4;
    for (int64_t row = int64_t(blockIdx.x) * RPP + rr; row < n; row += int64_t(gridDim.x) * RPP) {
        T acc[4] = {0, 0, 0, 0};
        for (int k = 0; k < nblk; ++k) {
            const T *p = basis + int64_t(k) * stride + row * W + c4;
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(som[k * W + c4 + q], p[q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (c4 + q < mo) Y[row * ldy + c4 + q] = acc[q];
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

// ---------------------------------------------------------------- launchers
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
    k_hkk<T><<<1, 256, 0, s>>>(G, M, W, Hd, C, ctrl);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::SMALL, s, 0, 0);
    return 0;
}

template <typename T>
int launch_chol(const double *G, int M, int W, int pass, int step, double inv_thresh2,
                double piv_rel2, double *R1, T *Rinv, double *Hs, T *Bout, Ctrl *ctrl,
                cudaStream_t s) {
    const size_t smem = sizeof(double) * (size_t(M) * (M + 1) + M);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_chol<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(sizeof(double) * (128 * 129 + 128)));
        attr = true;
    }
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

int launch_lanczos_alpha(const double *parts, int nparts, int W, int M, int gbl, int k,
                         const double *sigma, double *alpha, double *a_upd, const Ctrl *ctrl,
                         cudaStream_t s) {
    prof_begin(KernelClass::SMALL, s);
    k_lanczos_alpha<<<1, 256, 0, s>>>(parts, nparts, W, M, gbl, k, sigma, alpha, a_upd, ctrl);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::SMALL, s, double(nparts) * W * 8, 0);
    return 0;
}

int launch_lanczos_beta(const double *parts, int nparts, int W, int M, int gbl, int k, int round32,
                        double thresh, double *beta, double *sigma, int32_t *alive, double *c1,
                        double *c2, Ctrl *ctrl, cudaStream_t s) {
    prof_begin(KernelClass::SMALL, s);
    k_lanczos_beta<<<1, 256, 0, s>>>(parts, nparts, W, M, gbl, k, round32, thresh, beta, sigma,
                                     alive, c1, c2, ctrl);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::SMALL, s, double(nparts) * W * 8, 0);
    return 0;
}

int launch_tridiag_phi(int W, int M, int m, int gbl, const double *alpha, const double *beta,
                       const double *sigma, int phi_kind, double eps, int s_int, double lam,
                       const ChebCoef &cc, double *omega, double *work, const Ctrl *ctrl,
                       cudaStream_t s) {
    prof_begin(KernelClass::PROJECTED, s);
    k_tridiag_phi<<<(W + 63) / 64, 64, 0, s>>>(W, M, m, gbl, alpha, beta, sigma, phi_kind, eps,
                                                s_int, lam, cc, omega, work, ctrl);
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::PROJECTED, s, 0, 0);
    return 0;
}

template <typename T>
int launch_axpy_colnorm(int W, T *X, const T *P, const double *a, int64_t n, double *parts,
                        int *grid_out, const Ctrl *ctrl, cudaStream_t s) {
    const int rpp = 256 / (W / 4);
    const int grid = int(std::min<int64_t>((n + rpp - 1) / rpp, int64_t(num_sms()) * 4));
    *grid_out = std::max(grid, 1);
    prof_begin(KernelClass::ROWBLOCK, s);
    switch (W) {
        case 16: k_axpy_colnorm<T, 16><<<*grid_out, 256, 0, s>>>(X, P, a, n, parts, ctrl); break;
        case 32: k_axpy_colnorm<T, 32><<<*grid_out, 256, 0, s>>>(X, P, a, n, parts, ctrl); break;
        case 64: k_axpy_colnorm<T, 64><<<*grid_out, 256, 0, s>>>(X, P, a, n, parts, ctrl); break;
        case 128: k_axpy_colnorm<T, 128><<<*grid_out, 256, 0, s>>>(X, P, a, n, parts, ctrl); break;
        default: return fail(KB_ERR_ARG, "bad width");
    }
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::ROWBLOCK, s, 3.0 * double(n) * W * sizeof(T), 3.0 * double(n) * W);
    return 0;
}

int axpy_max_grid() { return num_sms() * 4; }

#define KB_ASM_DIAG(WW)                                                                       \
    do {                                                                                      \
        cudaFuncSetAttribute(k_assemble_diag<T, WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             int(smem));                                                      \
        k_assemble_diag<T, WW><<<grid, 256, smem, s>>>(basis, stride, nblk, omega, n, Y, ldy, mo); \
    } while (0)

template <typename T>
int launch_assemble_diag(int W, const T *basis, int64_t stride, int nblk, const double *omega,
                         int64_t n, float *Y, int64_t ldy, int mo, int64_t M_alg, cudaStream_t s) {
    const int rpp = 256 / (W / 4);
    const int grid = std::max(1, int(std::min<int64_t>((n + rpp - 1) / rpp, int64_t(num_sms()) * 8)));
    const size_t smem = sizeof(T) * size_t(nblk) * W;
    if (smem > 200 * 1024) return fail(KB_ERR_UNSUPPORTED, "too many blocks for the diagonal assembly");
    prof_begin(KernelClass::ASSEMBLE, s);
    switch (W) {
        case 16: KB_ASM_DIAG(16); break;
        case 32: KB_ASM_DIAG(32); break;
        case 64: KB_ASM_DIAG(64); break;
        case 128: KB_ASM_DIAG(128); break;
        default: return fail(KB_ERR_ARG, "bad width");
    }
    KB_CUDA_TRY(cudaGetLastError());
    prof_end(KernelClass::ASSEMBLE, s, double(nblk) * n * M_alg * sizeof(T) + double(n) * M_alg * 4,
             2.0 * nblk * double(n) * M_alg);
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
    template int launch_axpy_colnorm<T>(int, T *, const T *, const double *, int64_t, double *, \
                                        int *, const Ctrl *, cudaStream_t);                     \
    template int launch_assemble_diag<T>(int, const T *, int64_t, int, const double *, int64_t, \
                                         float *, int64_t, int, int64_t, cudaStream_t);         \
    template int launch_u_convert<T>(const double *, int, int, int, T *, const Ctrl *, cudaStream_t);
KB_INST(float)
KB_INST(double)
#undef KB_INST

}  // namespace kb
