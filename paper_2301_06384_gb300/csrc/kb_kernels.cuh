// Launchers of the small / element-wise / projected-problem kernels (internal).
#pragma once

#include <algorithm>

#include "kb_internal.cuh"

namespace kb {

// Up to CAP node indices passed by value to a kernel (no host-to-device copy needed).
struct NodeChunk {
    static constexpr int CAP = 256;
    int32_t idx[CAP];
    int32_t cnt;
    int32_t col0;
};

// Chebyshev coefficients d_0..d_{n-1} passed by value (sum_j d_j T_j, no halving).
struct ChebCoef {
    static constexpr int CAP = 440;
    int32_t n;
    double d[CAP];
};

// Rational (quadrature) form of the fractional spline power, used for non-integer s:
//   (eps + lambda)^{-s} = (eps + lambda)^{-s_int} * sum_k weight_k / (shift_k + lambda),
// s_int = floor(s); the sum approximates (eps + lambda)^{-alpha}, alpha = s - s_int, on
// [0, lam] by Gauss-Jacobi quadrature of the Stieltjes integral of z^{-alpha}
// (quadrature.cu).  n = 0 when s is an integer.  Passed to kernels by value.
struct QuadRule {
    static constexpr int CAP = 240;   // keeps the struct under 4 KB of kernel parameters
    int32_t n;
    int32_t s_int;
    double shift[CAP];
    double weight[CAP];
};
// Fills q for (eps, s) on the spectral interval [0, lam] such that the relative error of the
// sum on [0, lam] is at most tol (checked on a grid); KB_ERR_UNSUPPORTED when CAP nodes do
// not reach tol, KB_ERR_ARG for bad arguments.  Host only.
int spline_quadrature(double eps, double s, double lam, double tol, QuadRule &q);

// Coefficients of the projected step of gbl / sbl passed to the tridiagonal kernel: the
// Chebyshev series of e^{-t lambda} (diffusion kernel) or, for the spline kernel with
// non-integer s, the quadrature rule of the fractional power.
struct TriCoef {
    union {
        ChebCoef cc;
        QuadRule q;
    };
};
static_assert(sizeof(TriCoef) <= 3900, "projected-step coefficients must fit the 4 KB kernel parameter space");

int launch_ctrl_init(Ctrl *c, int steps, cudaStream_t s);
// dst = src with steps = min(src->steps, k) (the projected problem of the first k steps),
// or 0 once src stopped
int launch_ctrl_snapshot(Ctrl *dst, const Ctrl *src, int k, cudaStream_t s);
// Stopping rule of the serving workload: with steps = chk->steps and p = *prev_steps,
// stops ctrl (stop = 1, steps) when p > 0 and ||U - [Up; 0]||_F <= tol ||U||_F (U, Up:
// (steps M) x M and (p M) x M row-major); then *prev_steps = steps.  No-op once ctrl stopped.
// buf: index of U among the alternating check buffers; recorded in ctrl->from_check when the
// check stops the process.
int launch_conv_check(const double *U, const double *Up, int M, const Ctrl *chk, int32_t *prev_steps,
                      double tol, Ctrl *ctrl, cudaStream_t s, int buf);
// dst = src, with steps = 0 when src->from_check >= 0 (the final projected solve is then
// skipped); launch_copy_check_u copies that check's U (buffers of per doubles) into U.
int launch_ctrl_final(Ctrl *dst, const Ctrl *src, cudaStream_t s);
int launch_copy_check_u(const double *Uc, int64_t per, double *U, int M, int m, const Ctrl *ctrl,
                        cudaStream_t s);
template <typename T>
int launch_scatter(T *block, int64_t ld, const int32_t *nodes, int M, int col0, T val, cudaStream_t s);
int launch_marker(int32_t *marker, const int32_t *nodes, int M, cudaStream_t s);
template <typename T>
int launch_scale_copy(T *out, const T *in, int64_t count, double scale, cudaStream_t s);
int launch_fill_nan(float *Y, int64_t n, int64_t ldy, int mo, const Ctrl *ctrl, cudaStream_t s);

template <typename T>
int launch_hkk(const double *G, int M, int W, double *Hd, T *C, const Ctrl *ctrl, cudaStream_t s);
template <typename T>
int launch_chol(const double *G, int M, int W, int pass, int step, double inv_thresh2,
                double piv_rel2, double *R1, T *Rinv, double *Hs, T *Bout, Ctrl *ctrl,
                cudaStream_t s);

int launch_lanczos_init(int W, int M, int gbl, int round32, double *sigma, int32_t *alive,
                        double *c1, double *c2, cudaStream_t s);
int launch_lanczos_alpha(const double *parts, int nparts, int W, int M, int gbl, int k, int df,
                         const double *sigma, double *alpha, double *a_upd, const Ctrl *ctrl,
                         cudaStream_t s);
int launch_lanczos_beta(const double *parts, int nparts, int W, int M, int gbl, int k, int round32,
                        double thresh, double *beta, double *sigma, int32_t *alive, double *c1,
                        double *c2, Ctrl *ctrl, cudaStream_t s);
// phi(T) e_1 per tridiagonal T (one for gbl, one per column for sbl).  Spline kernel:
// (eps I + T)^{-s_int} applied after the fractional factor sum_k W_k (sigma_k I + T)^{-1}
// when tc.q.n > 0; qwork: 2 m tc.q.n doubles per column (nullptr when tc.q.n == 0).
// series: the full Chebyshev series of e^{-t lambda} (diffusion kernel); when it is longer
// than one ChebCoef it is applied in chunks (state in work, 4 m doubles per column) and tc.cc
// is not used.
int launch_tridiag_phi(int W, int M, int m, int gbl, const double *alpha, const double *beta,
                       const double *sigma, int phi_kind, double eps, int s_int, double lam,
                       const TriCoef &tc, double *omega, double *work, double *qwork, Ctrl *ctrl,
                       double bound, cudaStream_t s, const std::vector<double> *series = nullptr);
template <typename T>
int launch_axpy_colnorm(int W, T *X, const T *P, const double *a, int64_t n, double *parts,
                        int *grid_out, const Ctrl *ctrl, const int32_t *tgen, int limit,
                        int64_t M_alg, cudaStream_t s, const int32_t *alist = nullptr,
                        const int32_t *acount = nullptr);
int axpy_max_grid();
template <typename T>
int launch_assemble_diag(int W, const T *basis, int64_t stride, int nblk, const double *omega,
                         int64_t n, float *Y, int64_t ldy, int mo, int64_t M_alg,
                         const int32_t *tgen, cudaStream_t s, int kbase = 0, int accumulate = 0);

// Frontier restriction: hop distances from the node set (uint8, 255 = not reached) and
// per-32-row tile minima; expand(k) marks the rows at distance k.
int launch_frontier_init(uint8_t *gen, int32_t *tgen, int64_t n, const int32_t *nodes, int M,
                         cudaStream_t s);
// alist / acount (optional): the active-tile list of step k - 1 (launch_frontier_list with
// limit k - 1), which holds every row at distance k - 1; only those tiles are visited.
int launch_frontier_expand(const GraphDev &g, uint8_t *gen, int32_t *tgen, int k, cudaStream_t s,
                           const int32_t *alist = nullptr, const int32_t *acount = nullptr);
// Compacts the 32-row frontier tiles with tgen <= limit into list (increasing tile order,
// capacity ceil(n / 32)) and their number into *count; one CTA, deterministic.
int launch_frontier_list(const int32_t *tgen, int64_t n, int limit, int32_t *list, int32_t *count,
                         cudaStream_t s);
template <typename T>
int launch_u_convert(const double *U, int M, int W, int m, T *Ut, const Ctrl *ctrl, cudaStream_t s);

// Projected problem of the classical block Lanczos method (FP64, block tridiagonal H_m).
// Hdf: nullptr for the FP64 recurrence; else 2 m M^2 doubles of scratch for the split H, and
// the recurrence runs in double-float on the FP32 pipe (the FP32 and BF16 modes).
int launch_cheb_bt(const double *Hd, const double *Hs, int M, int m, double lam,
                   const std::vector<double> &d, double *V0, double *V1, double *V2, double *U,
                   const Ctrl *ctrl, cudaStream_t s, double *Hdf = nullptr);
// U = (eps I + H_m)^{-s} F_1.  Integer s: s_int block Cholesky solves (q == nullptr or
// q->n == 0).  Non-integer s: the quadrature rule q gives the fractional factor
// sum_k W_k (sigma_k I + H_m)^{-1} F_1, one block Cholesky factorisation and solve per node
// (qbatch nodes at a time, one CTA each, in qscr: qbatch * bt_quad_node_doubles(M, m)
// doubles), then s_int solves with eps I + H_m.  kmax: a host-side bound on ctrl->steps (the
// factorisation is launched block by block up to it; 0 means m).
__host__ __device__ inline size_t bt_quad_node_doubles(int M, int m) {
    return 3 * size_t(m) * M * M + size_t(m) * M;   // Ld, Ls, Y blocks and reciprocal diagonals
}
int launch_bt_spline(const double *Hd, const double *Hs, int M, int m, double eps, int s_int,
                     double *Ld, double *Ls, double *Yw, double *U, const Ctrl *ctrl,
                     cudaStream_t s, const QuadRule *q = nullptr, double *qscr = nullptr,
                     int qbatch = 0, int kmax = 0);

// Full reorthogonalisation: save the diagonal of the Gram of X before the first pass; after
// it, *skip = 1 when every column kept at least half of its squared norm (the second pass is
// then not needed).
int launch_reorth_save(const double *G, int M, int W, double *d0, cudaStream_t s);
int launch_reorth_decide(const double *G, const double *d0, int M, int W, int32_t *skip, cudaStream_t s);

// Graph utilities.
int launch_gershgorin(const GraphDev &g, double *out, cudaStream_t s);

// Marks the solve KB_ERR_ORTHOGONALITY when |U| exceeds bound or is NaN.
int launch_check_projected(const double *U, int64_t count, double bound, Ctrl *ctrl, cudaStream_t s);

}  // namespace kb
