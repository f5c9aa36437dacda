// Quadrature form of the fractional spline kernel (eps + lambda)^{-alpha}, 0 < alpha < 1,
// for the projected problems of the Lanczos methods with non-integer s (Section 2.4 defines
// the variational spline kernel for every s > 0; the projected step of Algorithms 1 and 2
// needs phi(H_m) F_1).
//
// For z > 0 and 0 < alpha < 1, z^{-alpha} is a Stieltjes function:
//     z^{-alpha} = (sin(pi alpha) / pi) * int_0^inf t^{-alpha} / (t + z) dt.
// Substituting t = c u^p, u = (1 - x) / (1 + x), x in (-1, 1), with the scale
// c = sqrt(eps (eps + lam)) (the geometric centre of [eps, eps + lam], where z = eps + lambda
// lies) and the stretch p = 3 gives
//     z^{-alpha} = (2 p sin(pi alpha) / pi) c^{1-alpha}
//                  * int_{-1}^{1} (1-x)^{p(1-alpha)-1} (1+x)^{p alpha-1} / (c (1-x)^p + z (1+x)^p) dx.
// The Jacobi weight (1-x)^{p(1-alpha)-1} (1+x)^{p alpha-1} takes the algebraic decay of both
// tails and is integrated exactly by Gauss-Jacobi quadrature (nodes x_k, weights w_k); what
// is left is smooth.  So
//     (eps + lambda)^{-alpha} ~ sum_k W_k / (sigma_k + lambda),
//     sigma_k = eps + c u_k^p > eps,   W_k = (2 p sin(pi alpha) / pi) c^{1-alpha} w_k / (1 + x_k)^p.
// Every shift is positive, so each term is an SPD solve with sigma_k I + H_m, whose spectrum
// lies in [0, lam].  The poles of the smooth factor sit where u^p = -z/c; the stretch p moves
// them away from the endpoints (distance of order ((eps + lam)/eps)^{-1/(2p)} instead of
// ((eps + lam)/eps)^{-1/2} for p = 1), so the error decays geometrically with a rate that
// depends only weakly on (eps + lam) / eps: about 60 nodes reach 1e-14 at (eps + lam)/eps = 3e6.
// The number of nodes is chosen by checking the rule against pow() on a grid of [0, lam].
//
// Gauss-Jacobi nodes and weights come from the Golub-Welsch method: the nodes are the
// eigenvalues of the symmetric tridiagonal Jacobi matrix of the three-term recurrence of the
// orthogonal polynomials of the weight, and the weights are mu_0 times the squared first
// components of its normalised eigenvectors.  The eigenproblem is solved by the implicit QL
// method with Wilkinson-type shifts, tracking only the first row of the eigenvector matrix.
#include "kb_internal.cuh"
#include "kb_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

namespace kb {
namespace {

// Implicit QL on the symmetric tridiagonal matrix with diagonal d[0..n) and off-diagonal
// e[0..n-1) (e[i] couples i and i+1).  On success d holds the eigenvalues and z the first
// components of the corresponding orthonormal eigenvectors (z starts as e_1).
bool tridiag_ql_first_row(std::vector<double> &d, std::vector<double> e, std::vector<double> &z) {
    const int n = int(d.size());
    e.resize(n, 0.0);
    z.assign(n, 0.0);
    z[0] = 1.0;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        while (true) {
            // smallest m >= l whose off-diagonal coupling to m + 1 is negligible
            int m = l;
            for (; m < n - 1; ++m) {
                const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= 1e-16 * dd) break;
            }
            if (m == l) break;
            if (++iter > 100) return false;
            // shift from the leading 2 x 2 block of the unreduced part
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + std::copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = m - 1;
            bool underflow = false;
            for (; i >= l; --i) {
                const double f = s * e[i];
                const double b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    underflow = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                // the same plane rotation on columns i, i + 1 of the eigenvector matrix
                const double zf = z[i + 1];
                z[i + 1] = s * z[i] + c * zf;
                z[i] = c * z[i] - s * zf;
            }
            if (underflow) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    return true;
}

// Gauss-Jacobi rule with N nodes for the weight (1-x)^a (1+x)^b on [-1, 1] (a, b > -1).
bool gauss_jacobi(int N, double a, double b, std::vector<double> &x, std::vector<double> &w) {
    std::vector<double> diag(N), off(std::max(N - 1, 0));
    const double ab = a + b;
    for (int k = 0; k < N; ++k) {
        if (k == 0) {
            diag[k] = (b - a) / (ab + 2.0);
        } else {
            const double t = 2.0 * k + ab;
            diag[k] = (b * b - a * a) / (t * (t + 2.0));
        }
    }
    for (int k = 1; k < N; ++k) {
        double beta;
        if (k == 1) {
            beta = 4.0 * (1.0 + a) * (1.0 + b) / ((2.0 + ab) * (2.0 + ab) * (3.0 + ab));
        } else {
            const double t = 2.0 * k + ab;
            beta = 4.0 * k * (k + a) * (k + b) * (k + ab) / (t * t * (t + 1.0) * (t - 1.0));
        }
        off[k - 1] = std::sqrt(beta);
    }
    const double mu0 = std::exp((ab + 1.0) * std::log(2.0) + std::lgamma(a + 1.0) + std::lgamma(b + 1.0) -
                                std::lgamma(ab + 2.0));
    std::vector<double> z;
    if (!tridiag_ql_first_row(diag, off, z)) return false;
    std::vector<int> order(N);
    for (int k = 0; k < N; ++k) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int i, int j) { return diag[i] < diag[j]; });
    x.resize(N);
    w.resize(N);
    for (int k = 0; k < N; ++k) {
        x[k] = diag[order[k]];
        w[k] = mu0 * z[order[k]] * z[order[k]];
    }
    return true;
}

// Largest relative error of the rule against pow() on a grid of [0, lam] that is dense near
// 0 (where the function varies fastest on the scale eps) and includes both ends.
double rule_error(const QuadRule &q, double eps, double alpha, double lam) {
    double worst = 0.0;
    const int G = 400;
    for (int g = 0; g <= G; ++g) {
        // points eps-geometric from 0 to lam, plus uniform ones
        const double f = double(g) / G;
        const double lg = (g == 0) ? 0.0 : eps * (std::pow((eps + lam) / eps, f) - 1.0);
        for (double lmb : {lg, lam * f}) {
            double sum = 0.0;
            for (int k = 0; k < q.n; ++k) sum += q.weight[k] / (q.shift[k] + lmb);
            const double ref = std::pow(eps + lmb, -alpha);
            worst = std::max(worst, std::fabs(sum - ref) / ref);
        }
    }
    return worst;
}

}  // namespace

int spline_quadrature(double eps, double s, double lam, double tol, QuadRule &q) {
    if (!(eps > 0) || !std::isfinite(eps) || !(s > 0) || !std::isfinite(s) || !(lam > 0) ||
        !std::isfinite(lam) || !(tol > 0))
        return fail(KB_ERR_ARG, "spline quadrature: bad eps, s, lambda or tol");
    const double fl = std::floor(s);
    q.s_int = int(fl);
    q.n = 0;
    const double alpha = s - fl;
    if (alpha == 0.0) return KB_OK;
    constexpr double P = 3.0;   // stretch of the substitution t = c u^P
    const double c = std::sqrt(eps * (eps + lam));
    const double pre = std::exp((1.0 - alpha) * std::log(c)) * 2.0 * P * std::sin(M_PI * alpha) / M_PI;
    std::vector<double> x, w;
    for (int N = 16;; N = std::min(QuadRule::CAP, N + N / 2)) {
        if (!gauss_jacobi(N, P * (1.0 - alpha) - 1.0, P * alpha - 1.0, x, w))
            return fail(KB_ERR_UNSUPPORTED, "spline quadrature: QL iteration did not converge");
        q.n = N;
        for (int k = 0; k < N; ++k) {
            const double op = 1.0 + x[k];
            const double u = (1.0 - x[k]) / op;
            q.shift[k] = eps + c * u * u * u;
            q.weight[k] = pre * w[k] / (op * op * op);
        }
        if (rule_error(q, eps, alpha, lam) <= tol) return KB_OK;
        if (N == QuadRule::CAP) break;
    }
    q.n = 0;
    return fail(KB_ERR_UNSUPPORTED, "spline quadrature: (eps + Lambda) / eps too large for " +
                                        std::to_string(QuadRule::CAP) + " quadrature nodes");
}

}  // namespace kb

extern "C" int kb_spline_quadrature(double eps, double s, double lam, double tol, double *shift,
                                    double *weight, int32_t cap, int32_t *count, int32_t *s_int) {
    try {
        if (!shift || !weight || !count || !s_int) return kb::fail(KB_ERR_ARG, "NULL argument");
        auto q = std::make_unique<kb::QuadRule>();
        const int rc = kb::spline_quadrature(eps, s, lam, tol, *q);
        if (rc) return rc;
        *count = q->n;
        *s_int = q->s_int;
        if (q->n > cap) return kb::fail(KB_ERR_ARG, "cap too small");
        for (int k = 0; k < q->n; ++k) {
            shift[k] = q->shift[k];
            weight[k] = q->weight[k];
        }
        return KB_OK;
    } catch (...) {
        return kb::fail(KB_ERR_CUDA, "unexpected exception");
    }
}
