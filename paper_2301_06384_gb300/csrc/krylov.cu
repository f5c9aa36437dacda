// The five block Krylov drivers and the kb_krylov_apply entry points.
//
//   cbl   Algorithm 1 (classical block Lanczos) with CholeskyQR2 for the reduced QR of
//         each new block and the FP64 projected problem U = phi(H_m) F_1.
//   gbl   Algorithm 2 (global block Lanczos), Frobenius inner products.
//   sbl   Section 3.3 (one ordinary Lanczos per column), run for all columns at once.
//   cheb  Section 3.4: the degree-m Lobatto interpolant applied by Clenshaw's backward
//         recurrence (same polynomial as the forward three-term recurrence; 3 block
//         reads/writes per product instead of 5).
//   cheb2 Section 3.4.1: the interpolant of sqrt(phi) of degree floor(m/2) applied twice.
//
// Every step runs on the device; the host only enqueues work.  No host synchronisation
// happens inside a solve (breakdown and early stops travel through a device control block).
#include "kb_internal.cuh"
#include "kb_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <mutex>

namespace kb {

// ---------------------------------------------------------------- host coefficient math
// e^{-t lambda} on [0, lam] as sum_k d_k T_k(1 - 2 lambda / lam):  with rho = t lam / 2,
// e^{-t lambda} = e^{-rho} e^{rho x} and e^{rho x} = I_0(rho) + 2 sum_k I_k(rho) T_k(x)
// (modified Bessel functions).  e^{-|rho|} I_k(|rho|) is computed by Miller's backward
// recurrence I_{k-1} = I_{k+1} + (2k/a) I_k, normalised by I_0 + 2 sum_k I_k = e^{a}.
std::vector<double> exp_series_coeffs(double t, double lam, double tol) {
    const double rho = 0.5 * t * lam;
    const double a = std::fabs(rho);
    if (a < 1e-300) return {1.0, 0.0};
    const int kmax = int(std::ceil(a + 12.0 * std::sqrt(a) + 60.0));
    std::vector<double> b(kmax + 2, 0.0);
    b[kmax + 1] = 0.0;
    b[kmax] = 1e-280;
    for (int k = kmax; k >= 1; --k) {
        b[k - 1] = b[k + 1] + (2.0 * k / a) * b[k];
        if (b[k - 1] > 1e250) {
            for (int q = k - 1; q <= kmax + 1; ++q) b[q] *= 1e-250;
        }
    }
    double S = b[0];
    for (int k = 1; k <= kmax; ++k) S += 2.0 * b[k];
    std::vector<double> d(kmax + 1);
    const double growth = rho < 0 ? std::exp(2.0 * a) : 1.0;
    double total = 0.0;
    for (int k = 0; k <= kmax; ++k) {
        double v = (k == 0 ? 1.0 : 2.0) * (b[k] / S) * growth;
        if (rho < 0 && (k & 1)) v = -v;
        d[k] = v;
        total += std::fabs(v);
    }
    int last = 1;
    for (int k = 0; k <= kmax; ++k)
        if (std::fabs(d[k]) > tol * total) last = std::max(last, k);
    d.resize(last + 1);
    return d;
}

// phi (or sqrt(phi)) at a point.
static double phi_value(kb_phi phi, const kb_params &p, double lam, bool sqrt_phi) {
    if (phi == KB_PHI_EXP) return std::exp(-(sqrt_phi ? 0.5 * p.t : p.t) * lam);
    return std::pow(p.eps + lam, -(sqrt_phi ? 0.5 * p.s : p.s));
}

// Eq. (chebcoeff) read as interpolation at the Chebyshev-Lobatto points:
//   c_k = (2/m) sum_{j=0..m}'' f(lambda_j) cos(pi j k / m),  lambda_j = lam/2 (1 - cos(pi j/m)),
// the double prime halving the j = 0 and j = m terms.  The series sum_k'' c_k T_k (c_0 and
// c_m halved) interpolates f on the grid.
// f and c: caller arrays of m + 1 doubles (f receives the samples); no allocation, so the
// fixed-scratch entry point shares it.
void lobatto_coeffs_into(kb_phi phi, const kb_params &p, int m, double lam, bool sqrt_phi, double *f,
                         double *c) {
    for (int j = 0; j <= m; ++j)
        f[j] = phi_value(phi, p, 0.5 * lam * (1.0 - std::cos(M_PI * j / m)), sqrt_phi);
    for (int k = 0; k <= m; ++k) {
        double s = 0.0;
        for (int j = 0; j <= m; ++j) {
            const double wj = (j == 0 || j == m) ? 0.5 : 1.0;
            // cos(pi j k / m) with the argument reduced mod 2m for accuracy
            const long r = (long(j) * k) % (2L * m);
            s += wj * f[j] * std::cos(M_PI * double(r) / m);
        }
        c[k] = 2.0 / m * s;
    }
}

std::vector<double> lobatto_coeffs(kb_phi phi, const kb_params &p, int m, double lam, bool sqrt_phi) {
    std::vector<double> f(m + 1), c(m + 1);
    lobatto_coeffs_into(phi, p, m, lam, sqrt_phi, f.data(), c.data());
    return c;
}

// The kernel choice and its parameters (Section 2.4): t finite for e^{-t lambda}; eps > 0 and
// s > 0, both finite, for (eps + lambda)^{-s}.
int validate_phi(kb_phi phi, const kb_params &p) {
    if (phi == KB_PHI_EXP) {
        if (!std::isfinite(p.t)) return fail(KB_ERR_ARG, "t not finite");
    } else if (phi == KB_PHI_SPLINE) {
        if (!(p.eps > 0) || !std::isfinite(p.eps)) return fail(KB_ERR_ARG, "eps must be > 0");
        if (!(p.s > 0) || !std::isfinite(p.s)) return fail(KB_ERR_ARG, "s must be > 0");
    } else {
        return fail(KB_ERR_ARG, "bad phi");
    }
    return KB_OK;
}

// ---------------------------------------------------------------- workspace
namespace {
struct Arena {
    char *base = nullptr;
    size_t off = 0;
    template <typename T>
    T *take(size_t count) {
        const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += bytes;
        return p;
    }
};

void ensure_pool(int dev) {
    // once per device; callers may run on several host threads (the serving workers)
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = std::numeric_limits<uint64_t>::max();
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done.push_back(dev);
}

struct Common {
    kb_graph *g;
    kb_phi phi;
    kb_params p;
    int s_int;
    cudaStream_t s;
    int spmm = 0;
    Ctrl *hctrl = nullptr;   // host copy of the control block when the caller wants info
    bool frontier = true;    // restrict the per-step kernels to the reached rows
    const QuadRule *quad = nullptr;   // spline kernel with non-integer s (Lanczos methods)
};

// The quadrature rule of the fractional spline power for the Lanczos methods (q->n = 0 when
// it is not needed: diffusion kernel, Chebyshev methods, integer s).  Relative accuracy
// 1e-14 on [0, Lambda], far below the FP64 rounding of the projected solves it feeds.
int quad_setup(const kb_graph *g, kb_method method, kb_phi phi, const kb_params &p, QuadRule &q) {
    q.n = 0;
    q.s_int = 0;
    if (phi != KB_PHI_SPLINE || method == KB_CHEB || method == KB_CHEB2) return KB_OK;
    return spline_quadrature(p.eps, p.s, g->lambda_proj, 1e-14, q);
}

// Quadrature nodes processed at once by the cbl projected step (one CTA and one scratch
// region of bt_quad_node_doubles(M, m) doubles each), at most 1 GiB of scratch.
int quad_batch(const QuadRule *q, int M, int m) {
    if (!q || q->n == 0) return 0;
    const size_t per = bt_quad_node_doubles(M, m) * sizeof(double);
    const size_t cap = std::max<size_t>(1, (size_t(1) << 30) / per);
    return int(std::min<size_t>({size_t(q->n), size_t(2 * num_sms()), cap}));
}
#define KB_TRY(x)                \
    do {                         \
        int _rc = (x);           \
        if (_rc) return _rc;     \
    } while (0)

// Largest |entry| of phi(H) F_1 when the spectrum of H lies in [0, Lambda] (F_1 = I on the
// first block): max phi on [0, Lambda]; infinity where no useful bound exists.
double projected_bound(const Common &c) {
    const double lam = c.g->lambda;
    if (c.phi == KB_PHI_EXP) {
        // slack 25 %: rounding of a slightly perturbed spectrum stays inside, a basis that
        // lost orthogonality (values growing like cosh(j acosh|x|), |x| > 1) does not
        if (c.p.t >= 0) return 1.25;
        const double e = -c.p.t * lam;
        return e < 700 ? std::exp(e) * 1.25 : std::numeric_limits<double>::infinity();
    }
    const double b = std::pow(c.p.eps, -c.p.s);
    return std::isfinite(b) ? b * 1.25 : std::numeric_limits<double>::infinity();
}

// ---------------------------------------------------------------- cbl
template <typename T>
struct CblBufs {
    using C = typename Cmp<T>::type;   // small matrices and Gram partials
    T *basis, *wbuf;
    C *parts, *Ut, *Cstk;
    // per-step small matrices (one W x W slot per step), kept for the two-pass replay:
    // H_kk as subtracted, H_{k,k+1} as subtracted at the next step, the two applied inverse
    // Cholesky factors, and the two local reorthogonalisation coefficient blocks
    C *Cbs, *Bs, *Rs1, *Rs2, *Cloc;
    double *Gsum, *Hd, *Hs, *R1, *V0, *V1, *V2, *U;
    double *Uc;          // stopping rule: two U_k of the checks (alternating)
    double *qscr;        // projected step with non-integer s: per-node block solves
    double *Hdf;         // projected e^{-tH} F_1 in double-float: H split into float pairs
    int32_t *chk_prev;   // steps of the previous check (0: none yet)
    double *reo_d0;      // full reorthogonalisation: squared column norms before the first pass
    int32_t *reo_skip;   // ... and the flag that skips the second pass
    Ctrl *ctrl, *ctrl2, *ctrl_chk;
    uint8_t *gen;
    int32_t *tgen;
    int32_t *alist, *acount;   // active 32-row tiles of the current step (frontier)
};

template <typename T>
void plan_cbl(Arena &ar, CblBufs<T> &b, int64_t n, int M, int W, int m, int rb_grid, bool two_pass,
              int qbatch) {
    b.basis = ar.take<T>(size_t(two_pass ? 3 : m) * n * W);
    b.wbuf = ar.take<T>(size_t(n) * W);
    using C = typename Cmp<T>::type;
    b.parts = ar.take<C>(size_t(rb_grid) * W * W);
    b.Cbs = ar.take<C>(size_t(m) * W * W * 6);   // Cbs | Bs | Rs1 | Rs2 | Cloc (2 per step)
    b.Bs = b.Cbs + size_t(m) * W * W;
    b.Rs1 = b.Bs + size_t(m) * W * W;
    b.Rs2 = b.Rs1 + size_t(m) * W * W;
    b.Cloc = b.Rs2 + size_t(m) * W * W;
    b.Ut = ar.take<C>(size_t(m) * W * W);
    b.Gsum = ar.take<double>(size_t(W) * W);
    b.Hd = ar.take<double>(size_t(m) * M * M);
    b.Hs = ar.take<double>(size_t(m) * M * M);
    b.R1 = ar.take<double>(size_t(M) * M);
    b.Cstk = ar.take<C>(size_t(m) * W * W);
    b.V0 = ar.take<double>(size_t(m) * M * M);
    b.V1 = ar.take<double>(size_t(m) * M * M);
    b.V2 = ar.take<double>(size_t(m) * M * M);
    b.U = ar.take<double>(size_t(m) * M * M);
    b.Uc = ar.take<double>(size_t(2) * m * M * M);
    b.qscr = qbatch > 0 ? ar.take<double>(size_t(qbatch) * bt_quad_node_doubles(M, m)) : nullptr;
    b.Hdf = sizeof(typename Cmp<T>::type) == 4 ? ar.take<double>(size_t(2) * m * M * M) : nullptr;
    b.chk_prev = ar.take<int32_t>(1);
    b.reo_d0 = ar.take<double>(size_t(W));
    b.reo_skip = ar.take<int32_t>(1);
    b.ctrl = ar.take<Ctrl>(1);
    b.ctrl2 = ar.take<Ctrl>(1);
    b.ctrl_chk = ar.take<Ctrl>(1);
    b.gen = ar.take<uint8_t>(size_t(n));
    b.tgen = ar.take<int32_t>(size_t((n + ACT_ROWS - 1) / ACT_ROWS));
    b.alist = ar.take<int32_t>(size_t((n + ACT_ROWS - 1) / ACT_ROWS));
    b.acount = ar.take<int32_t>(1);
}

template <typename T>
int run_cbl(Common &c, const int32_t *nodes, int M, int m, float *Y, int64_t ldy) {
    using C = typename Cmp<T>::type;
    const int64_t n = c.g->dev.n;
    const int W = width_for(M);
    const bool f64 = sizeof(C) == 8;
    const int rb_grid = rowblock_max_grid<T>(W);
    const bool two = c.p.two_pass != 0;
    const int qbatch = quad_batch(c.quad, M, m);
    Arena dry;
    CblBufs<T> b{};
    plan_cbl<T>(dry, b, n, M, W, m, rb_grid, two, qbatch);
    Arena ar;
    KB_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&ar.base), dry.off, c.s));
    plan_cbl<T>(ar, b, n, M, W, m, rb_grid, two, qbatch);
    auto body = [&]() -> int {
        const double lam = c.g->lambda;        // thresholds (scale of L)
        const double lam_p = c.g->lambda_proj; // interval of the projected series
        const double tau_inv = f64 ? 1e-12 : 1e-6;
        const double tau_piv = f64 ? 1e-12 : 1e-5;
        const double inv_thresh2 = (tau_inv * lam) * (tau_inv * lam) * M;
        const double piv2 = tau_piv * tau_piv;
        KB_TRY(launch_ctrl_init(b.ctrl, m, c.s));
        // with the frontier restriction only reached tiles are written, so every block
        // starts from zeros; otherwise each block is written in full
        const int nbuf = two ? 3 : m;
        KB_CUDA_TRY(cudaMemsetAsync(b.basis, 0, sizeof(T) * size_t(n) * W * (c.frontier ? nbuf : 1), c.s));
        KB_TRY(launch_scatter<T>(b.basis, W, nodes, M, 0, T(1), c.s));
        // slots of steps after a stop are never written: keep them zero
        KB_CUDA_TRY(cudaMemsetAsync(b.Cbs, 0, sizeof(C) * size_t(m) * W * W * 6, c.s));
        const int32_t *tg = c.frontier ? b.tgen : nullptr;
        if (c.frontier) {
            KB_TRY(launch_frontier_init(b.gen, b.tgen, n, nodes, M, c.s));
            KB_TRY(launch_frontier_list(b.tgen, n, 0, b.alist, b.acount, c.s));
            // the SpMM and the row-block kernels tile rows differently; rows of L Q_k that
            // the SpMM skips must read as zero in the row-block kernels (the reached set
            // only grows, so zeroing once suffices)
            KB_CUDA_TRY(cudaMemsetAsync(b.wbuf, 0, sizeof(T) * size_t(n) * W, c.s));
        }
        const int64_t bs = n * W;
        const size_t WW = size_t(W) * W;
        auto blk = [&](int j) { return b.basis + int64_t(two ? j % 3 : j) * bs; };
        int nchk = 0;
        if (c.p.tol > 0.0) KB_CUDA_TRY(cudaMemsetAsync(b.chk_prev, 0, sizeof(int32_t), c.s));
        for (int k = 1; k <= m; ++k) {
            T *Qk = blk(k - 1);
            T *Qp = k >= 2 ? blk(k - 2) : nullptr;
            C *Cb = b.Cbs + (k - 1) * WW;                     // H_kk
            const C *Bp = k >= 2 ? b.Bs + (k - 2) * WW : nullptr;   // H_{k-1,k} (step k-1)
            C *Bk = b.Bs + (k - 1) * WW;
            C *S1 = b.Rs1 + (k - 1) * WW, *S2 = b.Rs2 + (k - 1) * WW;
            C *Cl = b.Cloc + 2 * (k - 1) * WW;
            // Q_k is supported on rows within k-1 hops of W; L Q_k within k hops
            if (c.frontier) {
                KB_TRY(launch_frontier_expand(c.g->dev, b.gen, b.tgen, k, c.s, b.alist, b.acount));
                KB_TRY(launch_frontier_list(b.tgen, n, k, b.alist, b.acount, c.s));
            }
            // block SpMM: W = L Q_k
            LinEpi<T> e;
            e.s1 = 1.0;
            e.out = b.wbuf;
            e.ctrl = b.ctrl;
            e.tgen = tg;
            e.gen = tg ? b.gen : nullptr;
            e.limit = k;
            e.alist = tg ? b.alist : nullptr;
            e.acount = b.acount;
            KB_TRY(launch_spmm<T>(c.g->dev, W, Qk, e, c.s, nullptr, M, 0));
            ++c.spmm;
            // diagonal block: H_kk = Q_k^T L Q_k
            int grid = 0;
            RowArgs<T> pa;
            pa.n = n; pa.x = b.wbuf; pa.qa = Qk; pa.partials = b.parts; pa.ctrl = b.ctrl;
            pa.tgen = tg; pa.limit = k; pa.alist = tg ? b.alist : nullptr; pa.acount = b.acount;
            KB_TRY(launch_rowblock<T>(RB_PROJ, W, pa, c.s, &grid, M));
            KB_TRY(launch_reduce<C>(b.parts, grid, W * W, b.Gsum, c.s, b.ctrl));
            KB_TRY(launch_hkk<C>(b.Gsum, M, W, b.Hd + size_t(k - 1) * M * M, Cb, b.ctrl, c.s));
            if (k == m) break;   // Q_{m+1} is never used
            // three-term update: X = L Q_k - Q_{k-1} H_{k-1,k} - Q_k H_kk, then Gram X^T X
            T *X = blk(k);
            RowArgs<T> ua;
            ua.n = n; ua.x = b.wbuf; ua.qa = Qp; ua.ca = Bp; ua.qb = Qk; ua.cb = Cb;
            ua.out = X; ua.partials = b.parts; ua.ctrl = b.ctrl;
            ua.tgen = tg; ua.limit = k; ua.alist = tg ? b.alist : nullptr; ua.acount = b.acount;
            KB_TRY(launch_rowblock<T>(RB_UPD, W, ua, c.s, &grid, M));
            KB_TRY(launch_reduce<C>(b.parts, grid, W * W, b.Gsum, c.s, b.ctrl));
            if (c.p.reorth == 2) {
                // local reorthogonalisation (not in the paper): a second
                // classical Gram-Schmidt pass against Q_k and Q_{k-1},
                // X -= Q_k (Q_k^T X) + Q_{k-1} (Q_{k-1}^T X); it keeps the three-term
                // orthogonality that FP32 rounding erodes when Ritz values converge
                const T *loc[2] = {Qk, Qp};
                for (int j = 0; j < 2; ++j) {
                    if (!loc[j]) continue;
                    RowArgs<T> ra;
                    ra.n = n; ra.x = X; ra.qa = loc[j]; ra.partials = b.parts; ra.ctrl = b.ctrl;
                    ra.tgen = tg; ra.limit = k; ra.alist = tg ? b.alist : nullptr; ra.acount = b.acount;
                    KB_TRY(launch_rowblock<T>(RB_PROJ, W, ra, c.s, &grid, M));
                    KB_TRY(launch_reduce<C>(b.parts, grid, W * W, b.Gsum, c.s, b.ctrl, Cl + j * WW));
                }
                RowArgs<T> la;
                la.n = n; la.x = X; la.qa = Qp; la.ca = Cl + WW; la.qb = Qk;
                la.cb = Cl; la.out = X; la.partials = b.parts; la.ctrl = b.ctrl;
                la.tgen = tg; la.limit = k; la.alist = tg ? b.alist : nullptr; la.acount = b.acount;
                KB_TRY(launch_rowblock<T>(RB_UPD, W, la, c.s, &grid, M));
                KB_TRY(launch_reduce<C>(b.parts, grid, W * W, b.Gsum, c.s, b.ctrl));
            }
            if (c.p.reorth == 1) {
                // full reorthogonalisation (not in the paper): classical Gram-Schmidt against all
                // stored blocks, X -= Q_{1:k} (Q_{1:k}^T X); the second pass runs only when the
                // first removed more than half of some column's squared norm (Kahan's "twice
                // is enough"; the device decides, the host launches both passes); the last
                // subtraction that runs also forms the Gram X^T X for the QR
                KB_TRY(launch_reorth_save(b.Gsum, M, W, b.reo_d0, c.s));
                for (int pass = 0; pass < 2; ++pass) {
                    const int32_t *skip = pass == 1 ? b.reo_skip : nullptr;
                    for (int j = 0; j < k; ++j) {
                        RowArgs<T> ra;
                        ra.n = n; ra.x = X; ra.qa = b.basis + j * bs; ra.partials = b.parts;
                        ra.ctrl = b.ctrl; ra.skip = skip;
                        ra.tgen = tg; ra.limit = k; ra.alist = tg ? b.alist : nullptr; ra.acount = b.acount;
                        KB_TRY(launch_rowblock<T>(RB_PROJ, W, ra, c.s, &grid, M));
                        KB_TRY(launch_reduce<C>(b.parts, grid, W * W, b.Gsum, c.s, b.ctrl,
                                                b.Cstk + size_t(j) * W * W, skip));
                    }
                    RowArgs<T> sa;
                    sa.n = n; sa.x = X; sa.basis = b.basis; sa.block_stride = bs; sa.nblk = k;
                    sa.ca = b.Cstk; sa.out = X; sa.partials = b.parts; sa.ctrl = b.ctrl; sa.skip = skip;
                    sa.tgen = tg; sa.limit = k; sa.alist = tg ? b.alist : nullptr; sa.acount = b.acount;
                    KB_TRY(launch_rowblock<T>(RB_ASMSUB, W, sa, c.s, &grid, M));
                    KB_TRY(launch_reduce<C>(b.parts, grid, W * W, b.Gsum, c.s, b.ctrl, nullptr, skip));
                    if (pass == 0) KB_TRY(launch_reorth_decide(b.Gsum, b.reo_d0, M, W, b.reo_skip, c.s));
                }
            }
            // reduced QR: X = Q_{k+1} H_{k+1,k} by CholeskyQR2
            KB_TRY(launch_chol<C>(b.Gsum, M, W, 1, k, inv_thresh2, piv2, b.R1, S1, nullptr,
                                  nullptr, b.ctrl, c.s));
            RowArgs<T> ma;
            ma.n = n; ma.x = X; ma.ca = S1; ma.out = X; ma.partials = b.parts; ma.ctrl = b.ctrl;
            ma.tgen = tg; ma.limit = k; ma.alist = tg ? b.alist : nullptr; ma.acount = b.acount;
            KB_TRY(launch_rowblock<T>(RB_MULGRAM, W, ma, c.s, &grid, M));
            KB_TRY(launch_reduce<C>(b.parts, grid, W * W, b.Gsum, c.s, b.ctrl));
            KB_TRY(launch_chol<C>(b.Gsum, M, W, 2, k, inv_thresh2, piv2, b.R1, S2,
                                  b.Hs + size_t(k - 1) * M * M, Bk, b.ctrl, c.s));
            RowArgs<T> qa;
            qa.n = n; qa.x = X; qa.ca = S2; qa.out = X; qa.ctrl = b.ctrl;
            qa.tgen = tg; qa.limit = k; qa.alist = tg ? b.alist : nullptr; qa.acount = b.acount;
            KB_TRY(launch_rowblock<T>(RB_MUL, W, qa, c.s, &grid, M));
            // stopping rule: U_k at the check steps, compared with the previous check's
            if (c.p.tol > 0.0 && k < m && (k == 8 || k == 12 || k == 16 || k == 24 || k == 32 ||
                                           k == 48 || k == 64 || k == 96)) {
                double *Ucur = b.Uc + size_t(nchk % 2) * m * M * M;
                const double *Uprev = b.Uc + size_t((nchk + 1) % 2) * m * M * M;
                KB_TRY(launch_ctrl_snapshot(b.ctrl_chk, b.ctrl, k, c.s));
                if (c.phi == KB_PHI_EXP) {
                    const std::vector<double> d = exp_series_coeffs(c.p.t, lam_p, 1e-17);
                    KB_TRY(launch_cheb_bt(b.Hd, b.Hs, M, m, lam_p, d, b.V0, b.V1, b.V2, Ucur, b.ctrl_chk, c.s, b.Hdf));
                } else {
                    KB_TRY(launch_bt_spline(b.Hd, b.Hs, M, m, c.p.eps, c.s_int, b.V0, b.V1, b.V2, Ucur,
                                            b.ctrl_chk, c.s, c.quad, b.qscr, qbatch, k));
                }
                KB_TRY(launch_conv_check(Ucur, Uprev, M, b.ctrl_chk, b.chk_prev, c.p.tol, b.ctrl, c.s, nchk % 2));
                ++nchk;
            }
        }
        // projected problem: U = phi(H_m) F_1 in FP64 (skipped when the stopping rule's last
        // check formed it: the check's U is copied instead)
        const Ctrl *cfin = b.ctrl;
        if (c.p.tol > 0.0) {
            KB_TRY(launch_ctrl_final(b.ctrl_chk, b.ctrl, c.s));
            cfin = b.ctrl_chk;
        }
        if (c.phi == KB_PHI_EXP) {
            const std::vector<double> d = exp_series_coeffs(c.p.t, lam_p, 1e-17);
            KB_TRY(launch_cheb_bt(b.Hd, b.Hs, M, m, lam_p, d, b.V0, b.V1, b.V2, b.U, cfin, c.s, b.Hdf));
        } else {
            KB_TRY(launch_bt_spline(b.Hd, b.Hs, M, m, c.p.eps, c.s_int, b.V0, b.V1, b.V2, b.U,
                                    cfin, c.s, c.quad, b.qscr, qbatch));
        }
        if (c.p.tol > 0.0) KB_TRY(launch_copy_check_u(b.Uc, int64_t(m) * M * M, b.U, M, m, b.ctrl, c.s));
        KB_TRY(launch_check_projected(b.U, int64_t(m) * M * M, projected_bound(c), b.ctrl, c.s));
        KB_TRY(launch_u_convert<C>(b.U, M, W, m, b.Ut, b.ctrl, c.s));
        // assembly: Y = [Q_1 .. Q_m] U
        if (!two) {
            RowArgs<T> aa;
            aa.n = n; aa.basis = b.basis; aa.block_stride = bs; aa.nblk = m; aa.ca = b.Ut;
            aa.y = Y; aa.ldy = ldy; aa.mo = M; aa.ctrl = b.ctrl; aa.tgen = tg;
            int grid = 0;
            KB_TRY(launch_rowblock<T>(RB_ASM, W, aa, c.s, &grid, M));
        } else {
            // second pass: the same products and updates with the recorded matrices
            // (bit-identical blocks); Y += Q_k U_k as each block is recomputed
            KB_TRY(launch_ctrl_init(b.ctrl2, m, c.s));
            KB_CUDA_TRY(cudaMemsetAsync(b.basis, 0, sizeof(T) * size_t(n) * W * (c.frontier ? 3 : 1), c.s));
            KB_TRY(launch_scatter<T>(b.basis, W, nodes, M, 0, T(1), c.s));
            if (c.frontier) {
                KB_TRY(launch_frontier_init(b.gen, b.tgen, n, nodes, M, c.s));
                KB_TRY(launch_frontier_list(b.tgen, n, 0, b.alist, b.acount, c.s));
                KB_CUDA_TRY(cudaMemsetAsync(b.wbuf, 0, sizeof(T) * size_t(n) * W, c.s));
            }
            for (int k = 1; k <= m; ++k) {
                T *Qk = blk(k - 1);
                T *Qp = k >= 2 ? blk(k - 2) : nullptr;
                RowArgs<T> aa;
                aa.n = n; aa.basis = Qk; aa.block_stride = bs; aa.nblk = 1;
                aa.ca = b.Ut + (k - 1) * WW; aa.y = Y; aa.ldy = ldy; aa.mo = M; aa.tgen = tg;
                aa.kbase = k - 1; aa.accumulate = k > 1 ? 1 : 0;
                int grid = 0;
                KB_TRY(launch_rowblock<T>(RB_ASM, W, aa, c.s, &grid, M));
                if (k == m) break;
                if (c.frontier) {
                    KB_TRY(launch_frontier_expand(c.g->dev, b.gen, b.tgen, k, c.s, b.alist, b.acount));
                    KB_TRY(launch_frontier_list(b.tgen, n, k, b.alist, b.acount, c.s));
                }
                LinEpi<T> e;
                e.s1 = 1.0;
                e.out = b.wbuf;
                e.ctrl = b.ctrl2;
                e.tgen = tg;
                e.gen = tg ? b.gen : nullptr;
                e.limit = k;
                e.alist = tg ? b.alist : nullptr;
                e.acount = b.acount;
                KB_TRY(launch_spmm<T>(c.g->dev, W, Qk, e, c.s, nullptr, M, 0));
                ++c.spmm;
                T *X = blk(k);
                RowArgs<T> ua;
                ua.n = n; ua.x = b.wbuf; ua.qa = Qp; ua.ca = k >= 2 ? b.Bs + (k - 2) * WW : nullptr;
                ua.qb = Qk; ua.cb = b.Cbs + (k - 1) * WW;
                ua.out = X; ua.partials = b.parts; ua.ctrl = b.ctrl2; ua.tgen = tg; ua.limit = k; ua.alist = tg ? b.alist : nullptr; ua.acount = b.acount;
                KB_TRY(launch_rowblock<T>(RB_UPD, W, ua, c.s, &grid, M));
                if (c.p.reorth == 2) {
                    RowArgs<T> la = ua;
                    la.x = X; la.ca = b.Cloc + (2 * (k - 1) + 1) * WW; la.cb = b.Cloc + 2 * (k - 1) * WW;
                    KB_TRY(launch_rowblock<T>(RB_UPD, W, la, c.s, &grid, M));
                }
                for (int pass = 0; pass < 2; ++pass) {
                    RowArgs<T> qa;
                    qa.n = n; qa.x = X; qa.ca = (pass == 0 ? b.Rs1 : b.Rs2) + (k - 1) * WW;
                    qa.out = X; qa.ctrl = b.ctrl2; qa.tgen = tg; qa.limit = k; qa.alist = tg ? b.alist : nullptr; qa.acount = b.acount;
                    KB_TRY(launch_rowblock<T>(RB_MUL, W, qa, c.s, &grid, M));
                }
            }
        }
        KB_TRY(launch_fill_nan(Y, n, ldy, M, b.ctrl, c.s));
        return 0;
    };
    int rc = body();
    if (!rc && c.hctrl) {
        cudaError_t e = cudaMemcpyAsync(c.hctrl, b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c.s);
        if (e != cudaSuccess) rc = cuda_fail(e, "ctrl readback");
    }
    cudaFreeAsync(ar.base, c.s);
    return rc;
}

// ---------------------------------------------------------------- gbl / sbl
template <typename T>
struct LzBufs {
    T *basis;
    double *parts, *sigma, *alpha, *beta, *work;
    double *qwork;                    // fractional spline factor: 2 m nodes per column
    int32_t *alive;
    double *c1, *c2, *aupd, *omega;   // c1, c2, aupd: one row of W per step
    Ctrl *ctrl, *ctrl2;
    uint8_t *gen;
    int32_t *tgen;
    int32_t *alist, *acount;   // active 32-row tiles of the current step (frontier)
};

template <typename T>
void plan_lz(Arena &ar, LzBufs<T> &b, int64_t n, int W, int m, int pgrid, bool two_pass, int nquad) {
    // two-pass: three rotating blocks; the coefficients of every step are kept for the replay
    b.basis = ar.take<T>(size_t(two_pass ? 3 : m + 1) * n * W);
    b.parts = ar.take<double>(size_t(pgrid) * W);
    b.sigma = ar.take<double>(size_t(m + 1) * W);
    b.alpha = ar.take<double>(size_t(m + 1) * W);
    b.beta = ar.take<double>(size_t(m + 1) * W);
    b.work = ar.take<double>(size_t(W) * 4 * m);
    b.qwork = nquad > 0 ? ar.take<double>(size_t(W) * 2 * m * nquad) : nullptr;
    b.alive = ar.take<int32_t>(W);
    b.c1 = ar.take<double>(size_t(m + 1) * W);
    b.c2 = ar.take<double>(size_t(m + 1) * W);
    b.aupd = ar.take<double>(size_t(m + 1) * W);
    b.omega = ar.take<double>(size_t(m) * W);
    b.ctrl = ar.take<Ctrl>(1);
    b.ctrl2 = ar.take<Ctrl>(1);
    b.gen = ar.take<uint8_t>(size_t(n));
    b.tgen = ar.take<int32_t>(size_t((n + ACT_ROWS - 1) / ACT_ROWS));
    b.alist = ar.take<int32_t>(size_t((n + ACT_ROWS - 1) / ACT_ROWS));
    b.acount = ar.take<int32_t>(1);
}

template <typename T>
int run_lanczos_scalar(Common &c, bool gbl, const int32_t *nodes, int M, int m, float *Y,
                       int64_t ldy) {
    const int64_t n = c.g->dev.n;
    const int W = width_for(M);
    const bool f64 = sizeof(T) == 8;
    const int pgrid = std::max(spmm_max_grid<T>(W), axpy_max_grid());
    auto tc = std::make_unique<TriCoef>();
    int nquad = 0;
    std::vector<double> series;
    if (c.phi == KB_PHI_EXP) {
        series = exp_series_coeffs(c.p.t, c.g->lambda_proj, 1e-17);
        // longer series are applied in chunks by launch_tridiag_phi
        tc->cc.n = int(std::min<size_t>(series.size(), ChebCoef::CAP));
        for (int j = 0; j < tc->cc.n; ++j) tc->cc.d[j] = series[j];
    } else {
        tc->q.n = 0;
        tc->q.s_int = c.s_int;
        if (c.quad) {
            tc->q = *c.quad;
            nquad = c.quad->n;
        }
    }
    const bool two = c.p.two_pass != 0;
    Arena dry;
    LzBufs<T> b{};
    plan_lz<T>(dry, b, n, W, m, pgrid, two, nquad);
    Arena ar;
    KB_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&ar.base), dry.off, c.s));
    plan_lz<T>(ar, b, n, W, m, pgrid, two, nquad);
    auto body = [&]() -> int {
        const double thresh = (f64 ? 1e-12 : 1e-6) * c.g->lambda;
        KB_TRY(launch_ctrl_init(b.ctrl, m, c.s));
        const int nbuf = two ? 3 : m + 1;
        KB_CUDA_TRY(cudaMemsetAsync(b.basis, 0, sizeof(T) * size_t(n) * W * (c.frontier ? nbuf : 1), c.s));
        KB_TRY(launch_scatter<T>(b.basis, W, nodes, M, 0, T(1), c.s));
        const int32_t *tg = c.frontier ? b.tgen : nullptr;
        if (c.frontier) {
            KB_TRY(launch_frontier_init(b.gen, b.tgen, n, nodes, M, c.s));
            KB_TRY(launch_frontier_list(b.tgen, n, 0, b.alist, b.acount, c.s));
        }
        // coefficients of steps after an invariant stop are never written: keep them zero
        KB_CUDA_TRY(cudaMemsetAsync(b.c1, 0, sizeof(double) * size_t(m + 1) * W, c.s));
        KB_CUDA_TRY(cudaMemsetAsync(b.c2, 0, sizeof(double) * size_t(m + 1) * W, c.s));
        KB_CUDA_TRY(cudaMemsetAsync(b.aupd, 0, sizeof(double) * size_t(m + 1) * W, c.s));
        KB_CUDA_TRY(cudaMemsetAsync(b.beta, 0, sizeof(double) * size_t(m + 1) * W, c.s));
        KB_CUDA_TRY(cudaMemsetAsync(b.alpha, 0, sizeof(double) * size_t(m + 1) * W, c.s));
        KB_CUDA_TRY(cudaMemsetAsync(b.sigma, 0, sizeof(double) * size_t(m + 1) * W, c.s));
        KB_TRY(launch_lanczos_init(W, M, gbl ? 1 : 0, f64 ? 0 : 1, b.sigma, b.alive, b.c1, b.c2, c.s));
        const int64_t bs = n * W;
        auto blk = [&](int j) { return b.basis + int64_t(two ? j % 3 : j) * bs; };
        for (int k = 1; k <= m; ++k) {
            T *Pk = blk(k - 1);
            T *Pp = k >= 2 ? blk(k - 2) : nullptr;
            T *X = blk(k);
            if (c.frontier) {
                KB_TRY(launch_frontier_expand(c.g->dev, b.gen, b.tgen, k, c.s, b.alist, b.acount));
                KB_TRY(launch_frontier_list(b.tgen, n, k, b.alist, b.acount, c.s));
            }
            // X = L Q_k - h_{k,k-1} Q_{k-1}, with Q_k = sigma_k P_k; dots <P_k, X> per column
            LinEpi<T> e;
            e.tgen = tg;
            e.gen = tg ? b.gen : nullptr;
            e.limit = k;
            e.alist = tg ? b.alist : nullptr;
            e.acount = b.acount;
            e.a1 = b.c1 + int64_t(k - 1) * W;
            e.a2 = b.c2 + int64_t(k - 1) * W;
            e.s0 = 0.0;
            e.y = Pp;
            e.out = X;
            e.dot_partials = b.parts;
            e.ctrl = b.ctrl;
            int grid = 0;
            KB_TRY(launch_spmm<T>(c.g->dev, W, Pk, e, c.s, &grid, M, Pp ? 1 : 0));
            ++c.spmm;
            KB_TRY(launch_lanczos_alpha(b.parts, grid, W, M, gbl ? 1 : 0, k - 1, f64 ? 0 : 1, b.sigma, b.alpha,
                                        b.aupd + int64_t(k - 1) * W, b.ctrl, c.s));
            if (k == m) break;
            int grid2 = 0;
            KB_TRY(launch_axpy_colnorm<T>(W, X, Pk, b.aupd + int64_t(k - 1) * W, n, b.parts, &grid2,
                                          b.ctrl, tg, k, M, c.s, tg ? b.alist : nullptr, b.acount));
            KB_TRY(launch_lanczos_beta(b.parts, grid2, W, M, gbl ? 1 : 0, k - 1, f64 ? 0 : 1, thresh, b.beta,
                                       b.sigma, b.alive, b.c1 + int64_t(k) * W, b.c2 + int64_t(k) * W,
                                       b.ctrl, c.s));
        }
        KB_TRY(launch_tridiag_phi(W, M, m, gbl ? 1 : 0, b.alpha, b.beta, b.sigma, int(c.phi),
                                  c.p.eps, c.s_int, c.g->lambda_proj, *tc, b.omega, b.work, b.qwork, b.ctrl,
                                  projected_bound(c), c.s, c.phi == KB_PHI_EXP ? &series : nullptr));
        if (!two) {
            KB_TRY(launch_assemble_diag<T>(W, b.basis, bs, m, b.omega, n, Y, ldy, M, M, tg, c.s));
        } else {
            // second pass: the same products and updates with the recorded coefficients
            // (bit-identical blocks), each block added to Y as soon as it exists
            KB_TRY(launch_ctrl_init(b.ctrl2, m, c.s));
            KB_CUDA_TRY(cudaMemsetAsync(b.basis, 0, sizeof(T) * size_t(n) * W * (c.frontier ? 3 : 1), c.s));
            KB_TRY(launch_scatter<T>(b.basis, W, nodes, M, 0, T(1), c.s));
            if (c.frontier) {
                KB_TRY(launch_frontier_init(b.gen, b.tgen, n, nodes, M, c.s));
                KB_TRY(launch_frontier_list(b.tgen, n, 0, b.alist, b.acount, c.s));
            }
            KB_TRY(launch_assemble_diag<T>(W, blk(0), bs, 1, b.omega, n, Y, ldy, M, M, nullptr, c.s, 0, 0));
            for (int k = 1; k < m; ++k) {
                T *Pk = blk(k - 1);
                T *Pp = k >= 2 ? blk(k - 2) : nullptr;
                T *X = blk(k);
                if (c.frontier) {
                    KB_TRY(launch_frontier_expand(c.g->dev, b.gen, b.tgen, k, c.s, b.alist, b.acount));
                    KB_TRY(launch_frontier_list(b.tgen, n, k, b.alist, b.acount, c.s));
                }
                LinEpi<T> e;
                e.tgen = tg;
                e.gen = tg ? b.gen : nullptr;
                e.limit = k;
                e.alist = tg ? b.alist : nullptr;
                e.acount = b.acount;
                e.a1 = b.c1 + int64_t(k - 1) * W;
                e.a2 = b.c2 + int64_t(k - 1) * W;
                e.s0 = 0.0;
                e.y = Pp;
                e.out = X;
                e.dot_partials = b.parts;
                e.ctrl = b.ctrl2;
                int grid = 0;
                KB_TRY(launch_spmm<T>(c.g->dev, W, Pk, e, c.s, &grid, M, Pp ? 1 : 0));
                ++c.spmm;
                int grid2 = 0;
                KB_TRY(launch_axpy_colnorm<T>(W, X, Pk, b.aupd + int64_t(k - 1) * W, n, b.parts, &grid2,
                                              b.ctrl2, tg, k, M, c.s, tg ? b.alist : nullptr, b.acount));
                KB_TRY(launch_assemble_diag<T>(W, X, bs, 1, b.omega + int64_t(k) * W, n, Y, ldy, M, M,
                                               tg, c.s, k, 1));
            }
        }
        KB_TRY(launch_fill_nan(Y, n, ldy, M, b.ctrl, c.s));
        return 0;
    };
    int rc = body();
    if (!rc && c.hctrl) {
        cudaError_t e = cudaMemcpyAsync(c.hctrl, b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c.s);
        if (e != cudaSuccess) rc = cuda_fail(e, "ctrl readback");
    }
    cudaFreeAsync(ar.base, c.s);
    return rc;
}

// ---------------------------------------------------------------- cheb / cheb2
template <typename T>
int cheb_pass(Common &c, const std::vector<double> &coef, double lam, int W, int64_t n,
              const int32_t *marker, const int32_t *nodes, int Mc, const T *Zsrc, T *bufs[3],
              T *out, float *yout, int64_t ldo, int mo, int64_t M_alg, uint8_t *gen,
              int32_t *tgen, int hop0, int32_t *alist, int32_t *acount) {
    // weights of sum_k'' c_k T_k (Lobatto interpolation: c_0 and c_m halved)
    const int h = int(coef.size()) - 1;
    std::vector<double> w(coef);
    w[0] *= 0.5;
    w[h] *= 0.5;
    // b_h = w_h S
    int cur_i = 0, prev_i = -1;
    if (Zsrc) {
        KB_TRY(launch_scale_copy<T>(bufs[0], Zsrc, n * W, w[h], c.s));
    } else {
        KB_CUDA_TRY(cudaMemsetAsync(bufs[0], 0, sizeof(T) * size_t(n) * W, c.s));
        KB_TRY(launch_scatter<T>(bufs[0], W, nodes, Mc, 0, T(w[h]), c.s));
    }
    // b_k = w_k S + 2 A b_{k+1} - b_{k+2} (k = h-1..1);  result = w_0 S + A b_1 - b_2,
    // A = I - (2/lam) L
    for (int k = h - 1; k >= 0; --k) {
        const bool last = k == 0;
        int dst_i = 0;
        while (dst_i == cur_i || dst_i == prev_i) ++dst_i;
        // b_k is supported on rows within hop0 + (h - k) hops of W
        const int hop = hop0 + (h - k);
        if (tgen) {
            // the list of the previous hop holds every row at distance hop - 1; the list of
            // this hop serves this step's SpMM (the last step writes zeros on inactive tiles
            // and walks every tile) and the next expansion (the second cheb2 pass)
            KB_TRY(launch_frontier_expand(c.g->dev, gen, tgen, hop, c.s, alist, acount));
            KB_TRY(launch_frontier_list(tgen, n, hop, alist, acount, c.s));
        }
        LinEpi<T> e;
        e.tgen = tgen;
        e.gen = tgen ? gen : nullptr;
        e.limit = hop;
        e.alist = (tgen && !last) ? alist : nullptr;
        e.acount = acount;
        e.zero_inactive = last ? 1 : 0;
        e.s1 = (last ? -2.0 : -4.0) / lam;
        e.s0 = last ? 1.0 : 2.0;
        e.s2 = -1.0;
        e.y = prev_i >= 0 ? bufs[prev_i] : nullptr;
        if (Zsrc) { e.z = Zsrc; e.s3 = w[k]; }
        else { e.marker = marker; e.wE = w[k]; }
        if (last) {
            if (yout) e.yout = yout;
            else e.out = out;
        } else {
            e.out = bufs[dst_i];
        }
        KB_TRY(launch_spmm<T>(c.g->dev, W, bufs[cur_i], e, c.s, nullptr, M_alg,
                              (prev_i >= 0 ? 1 : 0) + (Zsrc ? 1 : 0), (last && yout) ? ldo : 0,
                              (last && yout) ? mo : 0));
        ++c.spmm;
        prev_i = cur_i;
        cur_i = dst_i;
    }
    return 0;
}

template <typename T>
void plan_cheb(Arena &ar, int64_t n, int Mmax, bool squared, T **bufs, T **Z, int32_t **marker,
               uint8_t **gen, int32_t **tgen, int32_t **alist, int32_t **acount) {
    const int Wmax = width_for(Mmax);
    for (int i = 0; i < 3; ++i) bufs[i] = ar.take<T>(size_t(n) * Wmax);
    *Z = squared ? ar.take<T>(size_t(n) * Wmax) : nullptr;
    *marker = ar.take<int32_t>(size_t(n));
    *gen = ar.take<uint8_t>(size_t(n));
    *tgen = ar.take<int32_t>(size_t((n + ACT_ROWS - 1) / ACT_ROWS));
    *alist = ar.take<int32_t>(size_t((n + ACT_ROWS - 1) / ACT_ROWS));
    *acount = ar.take<int32_t>(1);
}

template <typename T>
int run_cheb(Common &c, bool squared, const int32_t *nodes, int M, int m, float *Y, int64_t ldy) {
    const int64_t n = c.g->dev.n;
    const double lam = c.p.lambda_max > 0 ? c.p.lambda_max : c.g->lambda;
    const int h = squared ? m / 2 : m;
    const std::vector<double> coef = lobatto_coeffs(c.phi, c.p, h, lam, squared);
    const int Mmax = std::min(M, sizeof(T) == 8 ? 64 : 128);
    Arena dry;
    T *bufs[3], *Z;
    int32_t *marker, *tgen, *alist, *acount;
    uint8_t *gen;
    plan_cheb<T>(dry, n, Mmax, squared, bufs, &Z, &marker, &gen, &tgen, &alist, &acount);
    Arena ar;
    KB_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&ar.base), dry.off, c.s));
    plan_cheb<T>(ar, n, Mmax, squared, bufs, &Z, &marker, &gen, &tgen, &alist, &acount);
    auto body = [&]() -> int {
        for (int col0 = 0; col0 < M; col0 += Mmax) {
            const int Mc = std::min(Mmax, M - col0);
            const int W = width_for(Mc);
            KB_CUDA_TRY(cudaMemsetAsync(marker, 0xFF, sizeof(int32_t) * size_t(n), c.s));
            KB_TRY(launch_marker(marker, nodes + col0, Mc, c.s));
            int32_t *tg = nullptr;
            if (c.frontier) {
                // Clenshaw blocks are written on reached tiles only: start from zeros
                for (int i = 0; i < 3; ++i)
                    KB_CUDA_TRY(cudaMemsetAsync(bufs[i], 0, sizeof(T) * size_t(n) * W, c.s));
                if (Z) KB_CUDA_TRY(cudaMemsetAsync(Z, 0, sizeof(T) * size_t(n) * W, c.s));
                KB_TRY(launch_frontier_init(gen, tgen, n, nodes + col0, Mc, c.s));
                KB_TRY(launch_frontier_list(tgen, n, 0, alist, acount, c.s));
                tg = tgen;
            }
            if (!squared) {
                KB_TRY(cheb_pass<T>(c, coef, lam, W, n, marker, nodes + col0, Mc, nullptr, bufs,
                                    nullptr, Y + col0, ldy, Mc, Mc, gen, tg, 0, alist, acount));
            } else {
                KB_TRY(cheb_pass<T>(c, coef, lam, W, n, marker, nodes + col0, Mc, nullptr, bufs, Z,
                                    nullptr, 0, 0, Mc, gen, tg, 0, alist, acount));
                KB_TRY(cheb_pass<T>(c, coef, lam, W, n, marker, nodes + col0, Mc, Z, bufs,
                                    nullptr, Y + col0, ldy, Mc, Mc, gen, tg, h, alist, acount));
            }
        }
        return 0;
    };
    const int rc = body();
    cudaFreeAsync(ar.base, c.s);
    return rc;
}

// Scratch bytes of one solve (the same plans the runs allocate).
template <typename T>
size_t workspace_bytes_t(int64_t n, kb_method method, int M, int m, bool two, const QuadRule *q) {
    Arena dry;
    const int W = width_for(M);
    switch (method) {
        case KB_CBL: {
            CblBufs<T> b{};
            plan_cbl<T>(dry, b, n, M, W, m, rowblock_max_grid<T>(W), two, quad_batch(q, M, m));
            break;
        }
        case KB_GBL:
        case KB_SBL: {
            // sbl runs column groups one after the other; each group allocates its own scratch
            const int Mg = method == KB_SBL ? std::min(M, sizeof(T) == 8 ? 64 : 128) : M;
            const int Wg = width_for(Mg);
            LzBufs<T> b{};
            plan_lz<T>(dry, b, n, Wg, m, std::max(spmm_max_grid<T>(Wg), axpy_max_grid()), two,
                       q ? q->n : 0);
            break;
        }
        case KB_CHEB:
        case KB_CHEB2: {
            T *bufs[3], *Z;
            int32_t *marker, *tgen, *alist, *acount;
            uint8_t *gen;
            plan_cheb<T>(dry, n, std::min(M, sizeof(T) == 8 ? 64 : 128), method == KB_CHEB2, bufs, &Z,
                         &marker, &gen, &tgen, &alist, &acount);
            break;
        }
    }
    return dry.off;
}

}  // namespace
}  // namespace kb

// ---------------------------------------------------------------- C ABI
using namespace kb;

namespace {

int validate(kb_graph *g, kb_method method, kb_phi phi, const kb_params *params,
             const int32_t *nodes, int32_t M, int32_t m, const void *Y, int *s_int) {
    if (!g) return fail(KB_ERR_ARG, "graph is NULL");
    if (!params) return fail(KB_ERR_ARG, "params is NULL");
    if (!nodes) return fail(KB_ERR_ARG, "nodes is NULL");
    if (!Y) return fail(KB_ERR_ARG, "Y is NULL");
    if (method < KB_CBL || method > KB_CHEB2) return fail(KB_ERR_ARG, "bad method");
    if (M < 1 || M > g->dev.n) return fail(KB_ERR_ARG, "M out of range");
    if (m < 1 || m > 100000) return fail(KB_ERR_ARG, "m out of range");
    if (method == KB_CHEB2 && m < 2) return fail(KB_ERR_ARG, "KB_CHEB2 needs m >= 2");
    if (params->basis != KB_F32 && params->basis != KB_F64 && params->basis != KB_BF16)
        return fail(KB_ERR_ARG, "bad basis dtype");
    if (params->reorth < 0 || params->reorth > 2) return fail(KB_ERR_ARG, "reorth must be 0, 1 or 2");
    if (params->two_pass != 0 && params->two_pass != 1) return fail(KB_ERR_ARG, "two_pass must be 0 or 1");
    if (params->two_pass && params->reorth == 1)
        return fail(KB_ERR_UNSUPPORTED, "full reorthogonalisation needs the stored basis (two_pass = 0)");
    if (params->reorth && method != KB_CBL)
        return fail(KB_ERR_UNSUPPORTED, "reorthogonalisation is implemented for KB_CBL only");
    if (!(params->tol >= 0.0) || !std::isfinite(params->tol)) return fail(KB_ERR_ARG, "tol must be finite and >= 0");
    if (params->tol > 0.0 && method != KB_CBL)
        return fail(KB_ERR_UNSUPPORTED, "the stopping rule (tol > 0) is implemented for KB_CBL only");
    if (params->tol > 0.0 && params->two_pass)
        return fail(KB_ERR_UNSUPPORTED, "the stopping rule (tol > 0) needs the stored basis (two_pass = 0)");
    const int wmax = params->basis == KB_F64 ? 64 : 128;
    if ((method == KB_CBL || method == KB_GBL) && M > wmax)
        return fail(KB_ERR_UNSUPPORTED, "block width too large for this method and dtype");
    if (int rc = validate_phi(phi, *params)) return rc;
    *s_int = 0;
    if (phi == KB_PHI_SPLINE && (method == KB_CBL || method == KB_GBL || method == KB_SBL)) {
        // floor(s) block solves with eps I + H_m, the fractional rest by quadrature
        if (params->s >= 65) return fail(KB_ERR_UNSUPPORTED, "Lanczos methods support s < 65");
        *s_int = int(std::floor(params->s));
    }
    if (method == KB_CBL && phi == KB_PHI_EXP && std::fabs(params->t) * g->lambda_proj > 2e5)
        return fail(KB_ERR_UNSUPPORTED, "t * Lambda too large for the Chebyshev projected solve");
    std::vector<int32_t> sorted(nodes, nodes + M);
    std::sort(sorted.begin(), sorted.end());
    if (sorted.front() < 0 || sorted.back() >= g->dev.n) return fail(KB_ERR_NODES, "node index out of range");
    for (int i = 1; i < M; ++i)
        if (sorted[i] == sorted[i - 1]) return fail(KB_ERR_NODES, "repeated node " + std::to_string(sorted[i]));
    return KB_OK;
}

int apply_device(kb_graph *g, kb_method method, kb_phi phi, const kb_params *params,
                 const int32_t *nodes, int32_t M, int32_t m, float *Y, void *stream, kb_info *info) {
    int s_int = 0;
    int rc = validate(g, method, phi, params, nodes, M, m, Y, &s_int);
    if (rc) return rc;
    DeviceGuard dg;
    KB_CUDA_TRY(dg.set(g->device));
    ensure_pool(g->device);
    auto quad = std::make_unique<QuadRule>();
    rc = quad_setup(g, method, phi, *params, *quad);
    if (rc) return rc;
    Common c{g, phi, *params, s_int, static_cast<cudaStream_t>(stream), 0, nullptr, true};
    if (quad->n > 0) c.quad = quad.get();
    // exact restriction of the per-step kernels to rows reached from W (hop distances are
    // kept in 8 bits)
    c.frontier = !params->no_frontier && m <= FRONTIER_MAX_HOPS;
    const bool f64 = params->basis == KB_F64;
    const bool bf16 = params->basis == KB_BF16;
    const int chunk = f64 ? 64 : 128;
    // one host control block per column group (sbl may run several groups)
    std::vector<Ctrl> hc;
    const int ngroups = method == KB_SBL ? (M + chunk - 1) / chunk : 1;
    if (info) hc.assign(ngroups, Ctrl{KB_OK, 0, m, -1, -1.0, -1, 0});
    switch (method) {
        case KB_CBL:
            c.hctrl = info ? &hc[0] : nullptr;
            rc = f64 ? run_cbl<double>(c, nodes, M, m, Y, M)
                 : bf16 ? run_cbl<__nv_bfloat16>(c, nodes, M, m, Y, M)
                        : run_cbl<float>(c, nodes, M, m, Y, M);
            break;
        case KB_GBL:
            c.hctrl = info ? &hc[0] : nullptr;
            rc = f64 ? run_lanczos_scalar<double>(c, true, nodes, M, m, Y, M)
                 : bf16 ? run_lanczos_scalar<__nv_bfloat16>(c, true, nodes, M, m, Y, M)
                        : run_lanczos_scalar<float>(c, true, nodes, M, m, Y, M);
            break;
        case KB_SBL:
            for (int col0 = 0, gi = 0; col0 < M && !rc; col0 += chunk, ++gi) {
                const int Mc = std::min(chunk, M - col0);
                c.hctrl = info ? &hc[gi] : nullptr;
                rc = f64 ? run_lanczos_scalar<double>(c, false, nodes + col0, Mc, m, Y + col0, M)
                     : bf16 ? run_lanczos_scalar<__nv_bfloat16>(c, false, nodes + col0, Mc, m, Y + col0, M)
                            : run_lanczos_scalar<float>(c, false, nodes + col0, Mc, m, Y + col0, M);
            }
            break;
        case KB_CHEB:
        case KB_CHEB2:
            rc = f64 ? run_cheb<double>(c, method == KB_CHEB2, nodes, M, m, Y, M)
                 : bf16 ? run_cheb<__nv_bfloat16>(c, method == KB_CHEB2, nodes, M, m, Y, M)
                        : run_cheb<float>(c, method == KB_CHEB2, nodes, M, m, Y, M);
            break;
    }
    if (rc) return rc;
    if (!info) return KB_OK;
    KB_CUDA_TRY(cudaStreamSynchronize(c.s));
    info->status = KB_OK;
    info->steps_done = m;
    info->breakdown_step = -1;
    info->est_change = -1.0;
    for (const Ctrl &h : hc) {
        if (h.status != KB_OK) info->status = h.status;
        if (h.breakdown_step >= 0) info->breakdown_step = h.breakdown_step;
        if (method != KB_SBL) info->steps_done = h.steps;
    }
    if (method == KB_CBL && params->tol > 0.0) info->est_change = hc[0].est_change;
    if (method == KB_CHEB2) info->steps_done = 2 * (m / 2);
    info->spmm_launches = c.spmm;
    info->lambda_used = (method == KB_CHEB || method == KB_CHEB2)
                            ? (params->lambda_max > 0 ? params->lambda_max : g->lambda)
                            : 0.0;
    if (info->status == KB_ERR_ORTHOGONALITY)
        return fail(info->status, "the projected matrix left the spectral interval [0, Lambda] "
                                  "(loss of orthogonality of the Lanczos basis); use reorth");
    if (info->status == KB_ERR_CUDA)
        return fail(info->status, "a tensor-core kernel gave up waiting for its MMA completion");
    if (info->status != KB_OK) return fail(info->status, "Lanczos breakdown: rank-deficient block");
    return KB_OK;
}

}  // namespace

extern "C" int kb_krylov_apply(kb_graph *g, kb_method method, kb_phi phi, const kb_params *params,
                               const int32_t *nodes, int32_t M, int32_t m, float *Y, void *stream,
                               kb_info *info) {
    try {
        return apply_device(g, method, phi, params, nodes, M, m, Y, stream, info);
    } catch (const std::bad_alloc &) {
        return fail(KB_ERR_NOMEM, "host allocation failed");
    } catch (...) {
        return fail(KB_ERR_CUDA, "unexpected exception");
    }
}

extern "C" int kb_krylov_apply_host(kb_graph *g, kb_method method, kb_phi phi,
                                    const kb_params *params, const int32_t *nodes, int32_t M,
                                    int32_t m, float *Y_host, void *stream, kb_info *info) {
    try {
        if (!g || !Y_host) return fail(KB_ERR_ARG, "graph or Y_host is NULL");
        if (M < 1 || M > g->dev.n) return fail(KB_ERR_ARG, "M out of range");
        DeviceGuard dg;
        KB_CUDA_TRY(dg.set(g->device));
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        float *dY = nullptr;
        const size_t bytes = sizeof(float) * size_t(g->dev.n) * size_t(M);
        KB_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&dY), bytes, s));
        int rc = apply_device(g, method, phi, params, nodes, M, m, dY, stream, info);
        if (rc == KB_OK || rc == KB_ERR_BREAKDOWN) {
            cudaError_t e = cudaMemcpyAsync(Y_host, dY, bytes, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess && rc == KB_OK) rc = cuda_fail(e, "result copy");
        }
        cudaFreeAsync(dY, s);
        cudaStreamSynchronize(s);
        return rc;
    } catch (...) {
        return fail(KB_ERR_CUDA, "unexpected exception");
    }
}

extern "C" int kb_workspace_bytes(kb_graph *g, kb_method method, kb_phi phi, const kb_params *params,
                                  int32_t M, int32_t m, uint64_t *bytes) {
    try {
        if (!bytes) return fail(KB_ERR_ARG, "bytes is NULL");
        if (!g) return fail(KB_ERR_ARG, "graph is NULL");
        if (M < 1 || M > g->dev.n) return fail(KB_ERR_ARG, "M out of range");
        // validate everything but the node list (a dummy non-null list of distinct nodes)
        std::vector<int32_t> dummy(static_cast<size_t>(M));
        for (int i = 0; i < M; ++i) dummy[i] = i;
        int s_int = 0;
        const float probe = 0.f;
        int rc = validate(g, method, phi, params, dummy.data(), M, m, &probe, &s_int);
        if (rc) return rc;
        const int64_t n = g->dev.n;
        auto quad = std::make_unique<QuadRule>();
        rc = quad_setup(g, method, phi, *params, *quad);
        if (rc) return rc;
        const QuadRule *q = quad->n > 0 ? quad.get() : nullptr;
        const bool two = params->two_pass != 0;
        switch (params->basis) {
            case KB_F64: *bytes = workspace_bytes_t<double>(n, method, M, m, two, q); break;
            case KB_BF16: *bytes = workspace_bytes_t<__nv_bfloat16>(n, method, M, m, two, q); break;
            default: *bytes = workspace_bytes_t<float>(n, method, M, m, two, q); break;
        }
        return KB_OK;
    } catch (...) {
        return fail(KB_ERR_CUDA, "unexpected exception");
    }
}

extern "C" int kb_exp_series_coeffs(double t, double lam, double tol, double *d, int32_t cap,
                                    int32_t *count) {
    if (!d || !count || !(lam > 0)) return fail(KB_ERR_ARG, "bad argument");
    const std::vector<double> v = exp_series_coeffs(t, lam, tol);
    *count = int32_t(v.size());
    for (int i = 0; i < int(v.size()) && i < cap; ++i) d[i] = v[i];
    return int(v.size()) <= cap ? KB_OK : fail(KB_ERR_ARG, "cap too small");
}

extern "C" int kb_cheb_lobatto_coeffs(kb_phi phi, const kb_params *params, int32_t m, double lam,
                                      int32_t sqrt_phi, double *c) {
    if (!params || !c || m < 1 || !(lam > 0)) return fail(KB_ERR_ARG, "bad argument");
    const std::vector<double> v = lobatto_coeffs(phi, *params, m, lam, sqrt_phi != 0);
    for (int k = 0; k <= m; ++k) c[k] = v[k];
    return KB_OK;
}
