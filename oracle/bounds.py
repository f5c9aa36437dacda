"""A-priori error bounds of Section 4 (test infrastructure only).

Theorem 4.2: for the three Lanczos methods the error of the degree-p approximant is at
most 2 sqrt(N) E_p(phi); for the Chebyshev interpolant of degree m it is at most
sqrt(N) (2 + (2/pi) log(m+1)) E_m(phi).  Example 4.5, Eq. (boundapproximation), bounds
E_m(e^{-t lambda}) on [0, Lambda] explicitly (constants b and d as printed there; the
foci typo {0, Gamma} in Example 4.4 is read as {0, Lambda}).
"""
from __future__ import annotations

import math

B_CONST = (math.sqrt(5.0) - 1.0) / 2.0            # b ~ 0.618
D_CONST = (math.sqrt(5.0) - 2.0) * math.exp(B_CONST)  # d ~ 0.438


def best_approx_exp_bound(m: int, t: float, Lam: float) -> float:
    """Upper bound on E_m(e^{-t lambda}) over [0, Lambda], Eq. (boundapproximation)."""
    b, d = B_CONST, D_CONST
    tl = t * Lam
    if m <= tl:
        return (2.0 * math.exp(-b * (m + 1) ** 2 / tl) * (1.0 + math.sqrt(tl * math.pi / (4.0 * b)))
                + 2.0 * d ** tl / (1.0 - d))
    return 2.0 * d ** m / (1.0 - d)


def lanczos_error_bound(N: int, degree: int, t: float, Lam: float) -> float:
    """Theorem 4.2, Lanczos part: 2 sqrt(N) E_degree(phi) for phi = e^{-t lambda}."""
    return 2.0 * math.sqrt(N) * best_approx_exp_bound(degree, t, Lam)


def cheb_error_bound(N: int, m: int, t: float, Lam: float) -> float:
    """Theorem 4.2, Chebyshev part: sqrt(N)(2 + (2/pi) log(m+1)) E_m(phi)."""
    return math.sqrt(N) * (2.0 + 2.0 / math.pi * math.log(m + 1)) * best_approx_exp_bound(m, t, Lam)
