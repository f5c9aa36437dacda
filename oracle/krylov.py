"""FP64 block Krylov approximations of phi(L) E_W, step by step as the paper states them.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions
-----------
* ``L`` is a scipy.sparse CSR matrix in float64 holding the float32 CSR values promoted.
* ``m`` is the number of products with L (block SpMMs): the three Lanczos methods run
  k = 1..m of Algorithms 1/2 and return the degree m-1 polynomial p_{phi,m-1}; cheb
  returns the degree-m interpolant; cheb^2 squares the degree floor(m/2) interpolant of
  sqrt(phi) (so 2 floor(m/2) products).
* ``f`` is the scalar function phi (vectorised over numpy arrays).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .dense import unit_block


class Breakdown(RuntimeError):
    """A block of the Lanczos process became rank deficient.  The paper assumes full rank; a
    rank-deficient block is reported, not deflated."""


@dataclass
class KrylovResult:
    Y: np.ndarray                  # n x N approximation of phi(L) E_W
    steps: int                     # steps whose basis blocks enter the result
    H: np.ndarray | None = None    # the (block) Lanczos matrix H_m actually used
    basis: list = field(default_factory=list)


# ----------------------------------------------------------------------------- helpers
def laplacian(n: int, rowptr, col, val) -> sp.csr_matrix:
    """Sparse FP64 Laplacian from CSR (float32 values promoted exactly)."""
    return sp.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(col, dtype=np.int64),
                          np.asarray(rowptr, dtype=np.int64)), shape=(n, n))


def gershgorin_bound(L: sp.csr_matrix) -> float:
    """Lambda = max_i sum_j |L_ij|, an upper bound of the spectrum (Section 2.1 assumes a
    known bound Lambda; the Gershgorin bound is taken; it equals 2 max degree for D - A)."""
    return float(np.max(np.asarray(abs(L).sum(axis=1)).ravel()))


def matrix_function_sym(H: np.ndarray, f, F: np.ndarray) -> np.ndarray:
    """phi(H) F for a symmetric H through its spectral decomposition (the direct
    algorithm assumed in Section 7)."""
    Hs = 0.5 * (H + H.T)
    lam, V = np.linalg.eigh(Hs)
    return V @ (f(lam)[:, None] * (V.T @ F))


def _three_term(L, Qk, Qprev, Hprev_k):
    """Algorithm 1, three-term product: X = L Q_k - Q_{k-1} H_{k-1,k}, H_{k-1,k} = H_{k,k-1}^T (the symmetric block tridiagonal form)."""
    return L @ Qk - Qprev @ Hprev_k


def _project(Qk, X):
    """Algorithm 1, diagonal block: H_kk = Q_k^* X."""
    return Qk.T @ X


def _subtract(X, Qk, Hkk):
    """Algorithm 1, diagonal removal: X = X - Q_k H_kk."""
    return X - Qk @ Hkk


def _reorthogonalise(X, Q):
    """Full reorthogonalisation (not in the paper): classical Gram-Schmidt of
    X against every stored block Q_1..Q_k, X = X - [Q_1..Q_k]([Q_1..Q_k]^T X), applied twice
    (one pass leaves a component of relative size u * ||X_in|| / ||X_out|| along the basis
    when X is nearly inside its span; the second pass removes it)."""
    B = np.hstack(Q)
    for _ in range(2):
        X = X - B @ (B.T @ X)
    return X


def _reduced_qr(X):
    """Algorithm 1, reduced QR: X = Q_{k+1} H_{k+1,k}, H_{k+1,k} upper triangular.  The
    factor is fixed to a non-negative diagonal (the QR is unique only up to signs)."""
    Q, R = np.linalg.qr(X, mode="reduced")
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sgn[None, :], R * sgn[:, None]


# ----------------------------------------------------------------------------- cbl
def cbl(L: sp.csr_matrix, nodes, m: int, f, reorth: bool = False,
        tol: float = 1e-12) -> KrylovResult:
    """Classical block Lanczos, Algorithm 1.

    Q_1 = E_W; for k = 1..m: X = L Q_k - Q_{k-1} H_{k,k-1}^T; H_kk = Q_k^T X;
    X -= Q_k H_kk; (k < m) X = Q_{k+1} H_{k+1,k}.  Then U = phi(H_m) F_1 and
    Y = [Q_1..Q_m] U.  The QR at k = m is skipped because Q_{m+1} is unused.

    ``reorth`` (not in the paper): True or "full" subtracts Q_{1:k}(Q_{1:k}^T X)
    twice, right after the diagonal block is subtracted; "local" subtracts Q_k(Q_k^T X) + Q_{k-1}(Q_{k-1}^T X) once more
    (a second Gram-Schmidt pass against the two blocks of the three-term recurrence).  Breakdown: if X vanishes (||X||_F <= tol * Lambda * sqrt(N)) the block
    Krylov space is invariant, the process stops and H of the reached size is used (the
    result is then exact); a rank-deficient but non-zero X raises Breakdown.
    """
    n = L.shape[0]
    E = unit_block(n, nodes)
    N = E.shape[1]
    Lam = gershgorin_bound(L)
    Q = [E.copy()]
    Qprev = np.zeros_like(E)
    Hoff = np.zeros((N, N))          # H_{k,k-1}
    diag_blocks, sub_blocks = [], []
    steps = m
    for k in range(1, m + 1):
        Qk = Q[-1]
        X = _three_term(L, Qk, Qprev, Hoff.T)
        Hkk = _project(Qk, X)
        X = _subtract(X, Qk, Hkk)
        if reorth == "local":
            X = X - Qk @ (Qk.T @ X) - Qprev @ (Qprev.T @ X)
        elif reorth:
            X = _reorthogonalise(X, Q)
        diag_blocks.append(Hkk)
        if k == m:
            break
        if np.linalg.norm(X) <= tol * Lam * np.sqrt(N):
            steps = k
            break
        Qn, R = _reduced_qr(X)
        if np.min(np.abs(np.diag(R))) <= tol * Lam:
            raise Breakdown(f"rank-deficient block at step {k}")
        sub_blocks.append(R)
        Qprev, Hoff = Qk, R
        Q.append(Qn)
    H = np.zeros((steps * N, steps * N))
    for k in range(steps):
        H[k * N:(k + 1) * N, k * N:(k + 1) * N] = diag_blocks[k]
        if k + 1 < steps:
            R = sub_blocks[k]
            H[(k + 1) * N:(k + 2) * N, k * N:(k + 1) * N] = R
            H[k * N:(k + 1) * N, (k + 1) * N:(k + 2) * N] = R.T
    F1 = np.zeros((steps * N, N))
    F1[:N, :N] = np.eye(N)
    U = matrix_function_sym(H, f, F1)
    Y = np.hstack(Q[:steps]) @ U
    return KrylovResult(Y=Y, steps=steps, H=0.5 * (H + H.T), basis=Q[:steps])


# ----------------------------------------------------------------------------- gbl
def gbl(L: sp.csr_matrix, nodes, m: int, f, tol: float = 1e-12) -> KrylovResult:
    """Global block Lanczos, Algorithm 2 (Frobenius inner product).

    Q_1 = E_W / sqrt(N); X = L Q_k - h_{k-1,k} Q_{k-1}; h_kk = tr(Q_k^T X);
    X -= h_kk Q_k; h_{k+1,k} = ||X||_F; Q_{k+1} = X / h_{k+1,k}.
    u = sqrt(N) phi(H_m) f_1 and Y = sum_k u_k Q_k.  A vanishing X stops the process
    (invariant space)."""
    n = L.shape[0]
    E = unit_block(n, nodes)
    N = E.shape[1]
    Lam = gershgorin_bound(L)
    Q = [E / np.sqrt(N)]
    Qprev = np.zeros_like(E)
    hprev = 0.0
    alpha, beta = [], []
    steps = m
    for k in range(1, m + 1):
        Qk = Q[-1]
        X = L @ Qk - hprev * Qprev
        hkk = float(np.sum(Qk * X))           # tr(Q_k^T X)
        X = X - hkk * Qk
        alpha.append(hkk)
        if k == m:
            break
        h = float(np.linalg.norm(X))
        if h <= tol * Lam:
            steps = k
            break
        beta.append(h)
        Qprev, hprev = Qk, h
        Q.append(X / h)
    H = np.diag(alpha[:steps]) + np.diag(beta[:steps - 1], -1) + np.diag(beta[:steps - 1], 1)
    f1 = np.zeros((steps, 1))
    f1[0, 0] = 1.0
    u = np.sqrt(N) * matrix_function_sym(H, f, f1)[:, 0]
    Y = sum(u[k] * Q[k] for k in range(steps))
    return KrylovResult(Y=Y, steps=steps, H=H, basis=Q[:steps])


# ----------------------------------------------------------------------------- sbl
def sbl(L: sp.csr_matrix, nodes, m: int, f, tol: float = 1e-12) -> KrylovResult:
    """Sequential Lanczos (Section 3.3): an ordinary Lanczos run (Algorithm 1 or 2 with
    N = 1) on each column e_{w_i}; column i of the result is
    [q_1..q_m] phi(H_m^{(w_i)}) f_1 (the printed formula omits phi; it is applied here).  H is the
    block diagonal diag(H^{(w_1)}, ..., H^{(w_N)})."""
    nodes = np.asarray(nodes)
    cols, Hs = [], []
    for w in nodes:
        r = gbl(L, [w], m, f, tol=tol)
        cols.append(r.Y[:, 0])
        Hs.append(r.H)
    import scipy.linalg as sla
    return KrylovResult(Y=np.stack(cols, axis=1), steps=m, H=sla.block_diag(*Hs))


# ----------------------------------------------------------------------------- Chebyshev
def lobatto_nodes(m: int, Lam: float) -> np.ndarray:
    """lambda_j = Lambda/2 (1 - cos(pi j / m)), j = 0..m (Section 3.4)."""
    j = np.arange(m + 1)
    return 0.5 * Lam * (1.0 - np.cos(np.pi * j / m))


def cheb_coefficients(f, m: int, Lam: float) -> np.ndarray:
    """c_k(phi), k = 0..m, Eq. (chebcoeff) read as interpolation at the Chebyshev-Lobatto points:
    c_k = (2/m) sum_{j=0..m}'' phi(lambda_j) cos(pi j k / m), the sum halving the j = 0
    and j = m terms (equivalently the printed endpoint term with a minus sign)."""
    if m < 1:
        raise ValueError("m >= 1")
    lam = lobatto_nodes(m, Lam)
    fv = f(lam)
    w = np.ones(m + 1)
    w[0] = w[m] = 0.5
    j = np.arange(m + 1)
    C = np.cos(np.pi * np.outer(j, j) / m)     # C[k, j] = cos(pi j k / m)
    return (2.0 / m) * (C @ (w * fv))


def cheb_series_weights(m: int) -> np.ndarray:
    """Weights of Eq. (apprchebyshevseries) under the Lobatto reading: c_0 and c_m enter halved."""
    w = np.ones(m + 1)
    w[0] = w[m] = 0.5
    return w


def cheb_eval_scalar(c: np.ndarray, Lam: float, lam) -> np.ndarray:
    """p(lambda) = sum_k'' c_k T_k(1 - 2 lambda / Lambda), T_k(x) = cos(k arccos x)."""
    m = c.size - 1
    x = np.clip(1.0 - 2.0 * np.asarray(lam, dtype=np.float64) / Lam, -1.0, 1.0)
    k = np.arange(m + 1)
    T = np.cos(np.outer(np.arccos(x), k))
    return T @ (cheb_series_weights(m) * c)


def cheb_apply(L: sp.csr_matrix, B: np.ndarray, c: np.ndarray, Lam: float) -> np.ndarray:
    """sum_k'' c_k T_k(I - 2L/Lambda) B by the three-term recurrence
    T_{k+1} = 2 A T_k - T_{k-1}, T_0 = B, T_1 = A B (the recurrence applied to the block), A = I - (2/Lambda) L."""
    m = c.size - 1
    w = cheb_series_weights(m) * c
    A = lambda X: X - (2.0 / Lam) * (L @ X)
    T0 = B
    Y = w[0] * T0
    if m == 0:
        return Y
    T1 = A(T0)
    Y = Y + w[1] * T1
    for k in range(2, m + 1):
        T2 = 2.0 * A(T1) - T0
        Y = Y + w[k] * T2
        T0, T1 = T1, T2
    return Y


def cheb(L: sp.csr_matrix, nodes, m: int, f, Lam: float | None = None) -> KrylovResult:
    """Chebyshev interpolation method (Section 3.4): degree-m Lobatto interpolant of phi
    on [0, Lambda] applied to E_W by the three-term recurrence (m products with L)."""
    n = L.shape[0]
    Lam = gershgorin_bound(L) if Lam is None else float(Lam)
    c = cheb_coefficients(f, m, Lam)
    return KrylovResult(Y=cheb_apply(L, unit_block(n, nodes), c, Lam), steps=m)


def cheb2(L: sp.csr_matrix, nodes, m: int, fsqrt, Lam: float | None = None) -> KrylovResult:
    """Squared Chebyshev method (Section 3.4.1): p = (p^{cheb}_{sqrt(phi), floor(m/2)})^2,
    applied as two successive applications of the degree floor(m/2) interpolant of
    sqrt(phi) (2 floor(m/2) products with L)."""
    n = L.shape[0]
    Lam = gershgorin_bound(L) if Lam is None else float(Lam)
    h = m // 2
    if h < 1:
        raise ValueError("cheb2 needs m >= 2")
    c = cheb_coefficients(fsqrt, h, Lam)
    Z = cheb_apply(L, unit_block(n, nodes), c, Lam)
    return KrylovResult(Y=cheb_apply(L, Z, c, Lam), steps=2 * h)


# ----------------------------------------------------------------------------- dispatch
def apply(method: str, L: sp.csr_matrix, nodes, m: int, phi: str, t: float = 1.0,
          eps: float = 0.01, s: float = 1.0, reorth: bool = False,
          Lam: float | None = None) -> KrylovResult:
    """One entry for all five methods with the kernels of Section 2.4."""
    from .dense import phi_function, sqrt_phi_function
    f = phi_function(phi, t, eps, s)
    if method == "cbl":
        return cbl(L, nodes, m, f, reorth=reorth)
    if method == "gbl":
        return gbl(L, nodes, m, f)
    if method == "sbl":
        return sbl(L, nodes, m, f)
    if method == "cheb":
        return cheb(L, nodes, m, f, Lam)
    if method == "cheb2":
        return cheb2(L, nodes, m, sqrt_phi_function(phi, t, eps, s), Lam)
    raise ValueError(method)
