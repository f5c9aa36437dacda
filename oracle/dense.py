"""Dense FP64 spectral evaluation of kernel columns and textbook closed forms.

TEST INFRASTRUCTURE ONLY (see the package docstring).

phi(L) E_W is defined through the spectral decomposition L = V diag(lambda) V^T
(Section 2.4, "defined in terms of the spectral decomposition of L"; Section 3, the
naive two-step evaluation after Eq. (GBFcompute)): phi(L) E_W = V diag(phi(lambda)) V^T E_W.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------- kernels
def phi_function(phi: str, t: float = 1.0, eps: float = 0.01, s: float = 1.0):
    """The two kernels of Section 2.4: diffusion e^{-t lambda} and variational spline
    (eps + lambda)^{-s}; ``poly:c0,c1,...`` gives a test polynomial sum c_j lambda^j."""
    if phi == "exp":
        return lambda lam: np.exp(-t * np.asarray(lam, dtype=np.float64))
    if phi == "spline":
        return lambda lam: (eps + np.asarray(lam, dtype=np.float64)) ** (-s)
    if phi.startswith("poly:"):
        coeffs = [float(c) for c in phi[5:].split(",")]
        def p(lam):
            lam = np.asarray(lam, dtype=np.float64)
            out = np.zeros_like(lam)
            for c in reversed(coeffs):
                out = out * lam + c
            return out
        return p
    raise ValueError(phi)


def sqrt_phi_function(phi: str, t: float = 1.0, eps: float = 0.01, s: float = 1.0):
    """sqrt(phi) for the squared Chebyshev method (Section 3.4.1)."""
    if phi == "exp":
        return phi_function("exp", t=t / 2.0)
    if phi == "spline":
        return phi_function("spline", eps=eps, s=s / 2.0)
    f = phi_function(phi, t, eps, s)
    return lambda lam: np.sqrt(f(lam))


# ----------------------------------------------------------------------------- matrices
def laplacian_dense(n: int, rowptr, col, val) -> np.ndarray:
    """Dense FP64 copy of the CSR Laplacian (float32 values promoted exactly)."""
    L = np.zeros((n, n), dtype=np.float64)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr, dtype=np.int64)))
    L[rows, np.asarray(col, dtype=np.int64)] = np.asarray(val, dtype=np.float64)
    return L


def normalized_laplacian_dense(L: np.ndarray) -> np.ndarray:
    """I - D^{-1/2} A D^{-1/2} from a dense Laplacian (A = minus its off-diagonal part,
    D = weighted degrees; rows without edges stay zero).  The paper uses this Laplacian in
    Section 8 without a definition (read as the symmetric normalized Laplacian); its spectrum lies in [0, 2]."""
    A = -(L - np.diag(np.diag(L)))
    d = A.sum(axis=1)
    s = np.where(d > 0, 1.0 / np.sqrt(np.where(d > 0, d, 1.0)), 0.0)
    return np.diag((d > 0).astype(np.float64)) - (s[:, None] * A * s[None, :])


def unit_block(n: int, nodes) -> np.ndarray:
    """E_W = [e_{w_1}, ..., e_{w_N}] (Section 3)."""
    nodes = np.asarray(nodes, dtype=np.int64)
    E = np.zeros((n, nodes.size), dtype=np.float64)
    E[nodes, np.arange(nodes.size)] = 1.0
    return E


def kernel_columns(L: np.ndarray, nodes, f) -> np.ndarray:
    """phi(L) E_W = V diag(phi(lambda)) V^T E_W with V from a symmetric eigensolver."""
    lam, V = np.linalg.eigh(L)
    nodes = np.asarray(nodes, dtype=np.int64)
    return V @ (f(lam)[:, None] * V[nodes, :].T)


# ----------------------------------------------------------------------------- closed forms
def path_eigenpairs(n: int):
    """Path P_n (standard Laplacian): lambda_k = 2 - 2 cos(pi k / n) with eigenvectors
    v_k(i) = cos(pi k (i + 1/2) / n), k = 0..n-1 (the DCT-II basis), normalised."""
    k = np.arange(n)
    lam = 2.0 - 2.0 * np.cos(np.pi * k / n)
    i = np.arange(n)
    V = np.cos(np.pi * np.outer(i + 0.5, k) / n)
    V /= np.linalg.norm(V, axis=0)
    return lam, V


def cycle_eigenvalues(n: int) -> np.ndarray:
    """Cycle C_n: lambda_k = 2 - 2 cos(2 pi k / n), k = 0..n-1."""
    return 2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)


def path_function(n: int, f) -> np.ndarray:
    """f(L_path) from the closed-form eigenpairs (no eigensolver involved)."""
    lam, V = path_eigenpairs(n)
    return (V * f(lam)) @ V.T


def grid_exp_columns(dims, nodes, t: float) -> np.ndarray:
    """exp(-t L) E_W on a non-periodic grid with row-major numbering.  The grid Laplacian
    is the Kronecker sum of path Laplacians, so exp(-t L) is the Kronecker product of the
    path exponentials; each column is formed factor by factor from the closed form."""
    dims = [int(d) for d in dims]
    f = lambda lam: np.exp(-t * lam)
    factors = [path_function(d, f) for d in dims]
    nodes = np.asarray(nodes, dtype=np.int64)
    coords = np.unravel_index(nodes, dims)
    n = int(np.prod(dims))
    out = np.empty((n, nodes.size), dtype=np.float64)
    for c in range(nodes.size):
        col = np.ones(1)
        for ax, F in enumerate(factors):
            col = np.kron(col, F[:, coords[ax][c]])
        out[:, c] = col
    return out
