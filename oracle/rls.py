"""FP64 RLS kernel predictors from approximated kernel columns (Sections 2.3 and 5,
Algorithm 3).  TEST INFRASTRUCTURE ONLY (see the package docstring).

Given labels y at the sampling nodes W and kernel columns Y ~ phi(L) E_W, the RLS
coefficients solve (E_W^T Y + gamma N I) c = y (Eq. (computationcoefficientskrylov); with
the exact columns it is Eq. (computationcoefficients)), and the predictor on all nodes is
Y c.  For the classical block Lanczos method E_W^T Y = F_1^T phi(H_m) F_1 (proof of
Theorem 3.1), which is the matrix Algorithm 3 solves with; ``cbl_alg3`` forms it that way.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import dense, krylov


def coefficients(K: np.ndarray, y, gamma: float) -> np.ndarray:
    """c = (K + gamma N I)^{-1} y for the N x N collocation matrix K (a library dense solve,
    LU with partial pivoting)."""
    N = K.shape[0]
    return np.linalg.solve(K + gamma * N * np.eye(N), np.asarray(y, dtype=np.float64))


def predictor(Y: np.ndarray, nodes, y, gamma: float):
    """(predictor on all nodes, coefficients) from kernel columns Y (n x N)."""
    nodes = np.asarray(nodes, dtype=np.int64)
    c = coefficients(Y[nodes, :], y, gamma)
    return Y @ c, c


def exact(L: sp.csr_matrix, nodes, y, gamma: float, phi: str, **kw):
    """The RLS predictor with the exact kernel columns (dense spectral evaluation)."""
    Y = dense.kernel_columns(L.toarray(), nodes, dense.phi_function(phi, **kw))
    return predictor(Y, nodes, y, gamma)


def krylov_predictor(method: str, L: sp.csr_matrix, nodes, m: int, y, gamma: float, phi: str,
                     **kw):
    """The approximate predictor y^(kr) of Section 5 for one of the five methods."""
    Y = krylov.apply(method, L, nodes, m, phi, **kw).Y
    return predictor(Y, nodes, y, gamma)


def cbl_alg3(L: sp.csr_matrix, nodes, m: int, y, gamma: float, phi: str, **kw):
    """Algorithm 3 as printed: phi(H_m) F_1 and the basis from Algorithm 1, the system with
    F_1^T phi(H_m) F_1, the predictor [Q_1..Q_m] phi(H_m) F_1 c.  E_W has orthonormal
    columns, so its reduced QR is E_W = Q_1 F_1 with F_1 = I."""
    res = krylov.apply("cbl", L, nodes, m, phi, **kw)
    N = len(nodes)
    f = dense.phi_function(phi, **kw)
    H = res.H
    w, V = np.linalg.eigh(H)
    PhiF1 = (V * f(w)) @ V[:N, :].T           # phi(H_m) F_1 with F_1 = I (first N columns)
    c = coefficients(PhiF1[:N, :], y, gamma)
    Q = np.hstack(res.basis[: res.steps])
    return Q @ (PhiF1 @ c), c
