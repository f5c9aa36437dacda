"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each pin is independent of the oracle's own formulas: textbook closed forms, a library
matrix exponential, brute-force polynomial products, theorems of the paper (Theorem 3.1,
Proposition 3.2, the Lanczos exactness identity in the proof of Lemma 4.1, interpolation
at the Lobatto grid of Section 3.4, Theorem 4.2) and the paper's printed constants.  The
last group plants mistakes in the oracle and checks that a pin catches each one.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import bounds, dense, krylov

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _L(g):
    return krylov.laplacian(g.n, g.rowptr, g.col, g.val)


def _Ld(g):
    return dense.laplacian_dense(g.n, g.rowptr, g.col, g.val)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------------ dense oracle pins
@pytest.mark.parametrize("n", [2, 7, 50])
def test_path_spectrum_closed_form(n):
    lam = np.linalg.eigvalsh(_Ld(synth.path_graph(n)))
    ref = np.sort(2.0 - 2.0 * np.cos(np.pi * np.arange(n) / n))
    assert np.max(np.abs(lam - ref)) < 1e-12


@pytest.mark.parametrize("n", [3, 8, 41])
def test_cycle_spectrum_closed_form(n):
    lam = np.linalg.eigvalsh(_Ld(synth.cycle_graph(n)))
    assert np.max(np.abs(lam - np.sort(dense.cycle_eigenvalues(n)))) < 1e-12


@pytest.mark.parametrize("phi,kw", [("exp", dict(t=3.0)), ("spline", dict(eps=0.05, s=2.0))])
def test_path_kernel_matches_closed_form(phi, kw):
    n = 33
    g = synth.path_graph(n)
    f = dense.phi_function(phi, **kw)
    nodes = [0, 16, 32, 5]
    Y = dense.kernel_columns(_Ld(g), nodes, f)
    ref = dense.path_function(n, f)[:, nodes]
    assert np.max(np.abs(Y - ref)) < 1e-12


@pytest.mark.parametrize("dims", [(4, 5), (3, 3, 4), (32, 32)])
def test_grid_kronecker_closed_form(dims):
    g = synth.grid_graph(dims)
    nodes = synth.sample_nodes(g.n, 5, seed=2)
    Y = dense.kernel_columns(_Ld(g), nodes, dense.phi_function("exp", t=1.0))
    ref = dense.grid_exp_columns(dims, nodes, 1.0)
    assert np.max(np.abs(Y - ref)) < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_dense_matches_library_expm_and_solve(seed):
    g = synth.random_weighted_graph(40, 0.15, seed=seed)
    L = _Ld(g)
    nodes = synth.sample_nodes(g.n, 6, seed=seed)
    Y = dense.kernel_columns(L, nodes, dense.phi_function("exp", t=0.7))
    ref = sla.expm(-0.7 * L)[:, nodes]
    assert np.max(np.abs(Y - ref)) < 1e-12
    Y2 = dense.kernel_columns(L, nodes, dense.phi_function("spline", eps=0.1, s=2.0))
    A = 0.1 * np.eye(g.n) + L
    ref2 = np.linalg.solve(A, np.linalg.solve(A, dense.unit_block(g.n, nodes)))
    assert _rel(Y2, ref2) < 1e-11


def test_diffusion_column_sums_are_one():
    g = synth.random_geometric_graph(300, 8, seed=3)
    Y = dense.kernel_columns(_Ld(g), synth.sample_nodes(g.n, 7, 1), dense.phi_function("exp", t=2.0))
    assert np.max(np.abs(Y.sum(axis=0) - 1.0)) < 1e-12


def test_kernel_symmetric_positive_definite():
    g = synth.random_weighted_graph(30, 0.2, seed=5)
    nodes = np.arange(g.n)
    K = dense.kernel_columns(_Ld(g), nodes, dense.phi_function("spline", eps=0.01, s=1.0))
    assert np.max(np.abs(K - K.T)) < 1e-10
    assert np.min(np.linalg.eigvalsh(0.5 * (K + K.T))) > 0


# ------------------------------------------------------------------ Krylov oracle pins
def _poly_apply(L, nodes, coeffs):
    """sum_j c_j L^j E_W by repeated sparse products (brute force)."""
    E = dense.unit_block(L.shape[0], nodes)
    out = np.zeros_like(E)
    P = E
    for c in coeffs:
        out = out + c * P
        P = L @ P
    return out


@pytest.mark.parametrize("method", ["cbl", "gbl", "sbl"])
def test_lanczos_exact_for_low_degree_polynomials(method):
    # L^j E_W = Q H^j F_1 for j <= m-1 (proof of Lemma 4.1): exact for degree < m
    g = synth.random_geometric_graph(400, 9, seed=4)
    L = _L(g)
    nodes = synth.sample_nodes(g.n, 6, seed=1)
    coeffs = [1.0, 0.3, 0.02, 0.001]
    r = krylov.apply(method, L, nodes, 4, "poly:" + ",".join(map(str, coeffs)))
    assert _rel(r.Y, _poly_apply(L, nodes, coeffs)) < 1e-12
    # one degree more than the space holds is not reproduced: the pin is sensitive
    coeffs5 = coeffs + [1e-4]
    r5 = krylov.apply(method, L, nodes, 4, "poly:" + ",".join(map(str, coeffs5)))
    assert _rel(r5.Y, _poly_apply(L, nodes, coeffs5)) > 1e-8


def test_cbl_exact_at_full_dimension():
    # m N = n without breakdown: the Krylov space is R^n and the projection is exact
    g = synth.random_weighted_graph(12, 0.5, seed=7)
    nodes = [0, 5, 9]
    f = dense.phi_function("exp", t=0.8)
    r = krylov.cbl(_L(g), nodes, 4, f)
    assert _rel(r.Y, dense.kernel_columns(_Ld(g), nodes, f)) < 1e-10


def test_lanczos_exact_on_path_from_end_node():
    # single vector, m = n: distinct eigenvalues and nonzero end components => exact
    n = 16
    g = synth.path_graph(n)
    f = dense.phi_function("spline", eps=0.2, s=2.0)
    ref = dense.path_function(n, f)[:, [0]]
    for method in ["cbl", "gbl", "sbl"]:
        r = krylov.apply(method, _L(g), [0], n, "spline", eps=0.2, s=2.0)
        assert _rel(r.Y, ref) < 1e-9, method


def test_invariant_subspace_stops_early_and_is_exact():
    # nodes covering a whole connected component: the block space is invariant at once
    g = synth.from_edges(6, np.array([0, 1, 3]), np.array([1, 2, 4]))
    f = dense.phi_function("exp", t=1.0)
    r = krylov.cbl(_L(g), [0, 1, 2], 5, f)
    assert r.steps == 1
    assert _rel(r.Y, dense.kernel_columns(_Ld(g), [0, 1, 2], f)) < 1e-12


@pytest.mark.parametrize("phi,kw", [("exp", dict(t=5.0)), ("spline", dict(eps=0.01, s=2.0))])
@pytest.mark.parametrize("m", [1, 2, 3, 6])
def test_cbl_collocation_spd(phi, kw, m):
    # Theorem 3.1: E_W^T p^{cbl}(L) E_W is symmetric positive definite for every m
    g = synth.random_geometric_graph(500, 10, seed=8)
    nodes = synth.sample_nodes(g.n, 12, seed=3)
    r = krylov.apply("cbl", _L(g), nodes, m, phi, **kw)
    C = r.Y[nodes, :]
    assert np.max(np.abs(C - C.T)) < 1e-12 * np.max(np.abs(C))
    assert np.min(np.linalg.eigvalsh(0.5 * (C + C.T))) > 0


def test_cbl_ritz_values_in_spectrum_interval():
    # interlacing (proof of Theorem 3.1): spec(H_m) inside [0, Lambda]
    g = synth.random_geometric_graph(500, 10, seed=8)
    L = _L(g)
    r = krylov.apply("cbl", L, synth.sample_nodes(g.n, 8, 2), 6, "exp", t=1.0)
    lam = np.linalg.eigvalsh(r.H)
    lmax = np.linalg.eigvalsh(_Ld(g))[-1]
    assert lam.min() > -1e-10 and lam.max() < lmax + 1e-10


@pytest.mark.parametrize("method", ["gbl", "cheb"])
def test_collocation_symmetric(method):
    # Proposition 3.2 (gbl) and Section 3.4 (cheb): the polynomial is scalar, so symmetric
    g = synth.random_geometric_graph(500, 10, seed=9)
    nodes = synth.sample_nodes(g.n, 10, seed=4)
    r = krylov.apply(method, _L(g), nodes, 5, "exp", t=20.0)
    C = r.Y[nodes, :]
    assert np.max(np.abs(C - C.T)) < 1e-12 * np.max(np.abs(C))


def test_sbl_column_is_single_vector_cbl():
    g = synth.random_geometric_graph(400, 9, seed=10)
    L = _L(g)
    nodes = synth.sample_nodes(g.n, 5, seed=5)
    f = dense.phi_function("exp", t=2.0)
    Y = krylov.sbl(L, nodes, 7, f).Y
    for i, w in enumerate(nodes):
        assert _rel(Y[:, [i]], krylov.cbl(L, [w], 7, f).Y) < 1e-12


def test_block_size_one_all_lanczos_equal():
    g = synth.random_geometric_graph(400, 9, seed=11)
    L = _L(g)
    outs = [krylov.apply(mth, L, [17], 9, "spline", eps=0.05, s=2.0).Y for mth in ["cbl", "gbl", "sbl"]]
    assert _rel(outs[1], outs[0]) < 1e-12 and _rel(outs[2], outs[0]) < 1e-12


@pytest.mark.parametrize("m", [1, 2, 5, 16])
def test_cheb_interpolates_on_lobatto_grid(m):
    # Section 3.4: p^{cheb}_{phi,m} interpolates phi on the dilated Chebyshev-Lobatto grid
    Lam = 13.0
    f = dense.phi_function("exp", t=0.4)
    c = krylov.cheb_coefficients(f, m, Lam)
    lam = krylov.lobatto_nodes(m, Lam)
    assert np.max(np.abs(krylov.cheb_eval_scalar(c, Lam, lam) - f(lam))) < 1e-13


def test_cheb_exact_for_polynomials_up_to_degree_m():
    g = synth.random_geometric_graph(300, 9, seed=12)
    L = _L(g)
    nodes = synth.sample_nodes(g.n, 4, seed=6)
    coeffs = [0.5, 0.2, 0.03, 0.001]
    r = krylov.apply("cheb", L, nodes, 3, "poly:" + ",".join(map(str, coeffs)))
    assert _rel(r.Y, _poly_apply(L, nodes, coeffs)) < 1e-12


@pytest.mark.parametrize("method", ["cheb", "cheb2"])
def test_cheb_column_sums_equal_phi0(method):
    # L 1 = 0 for D - A, lambda = 0 is a grid node, so 1^T p(L) e_w = p(0) = phi(0)
    g = synth.random_geometric_graph(300, 9, seed=13)
    nodes = synth.sample_nodes(g.n, 6, seed=7)
    r = krylov.apply(method, _L(g), nodes, 10, "spline", eps=0.1, s=2.0)
    assert np.max(np.abs(r.Y.sum(axis=0) - 0.1 ** -2.0)) < 1e-10


def test_cheb2_collocation_psd():
    # Section 3.4.1: the squared polynomial is non-negative, so the collocation is PSD
    g = synth.random_geometric_graph(500, 10, seed=14)
    nodes = synth.sample_nodes(g.n, 20, seed=8)
    r = krylov.apply("cheb2", _L(g), nodes, 6, "exp", t=20.0)
    C = r.Y[nodes, :]
    assert np.min(np.linalg.eigvalsh(0.5 * (C + C.T))) > -1e-12


@pytest.mark.parametrize("t", [0.5, 2.0, 8.0])
@pytest.mark.parametrize("m", [4, 8, 14])
def test_theorem_4_2_bounds_hold(t, m):
    n = 60
    g = synth.path_graph(n)
    L = _L(g)
    Lam = krylov.gershgorin_bound(L)
    nodes = [0, 30, 59]
    ref = dense.path_function(n, dense.phi_function("exp", t=t))[:, nodes]
    for method in ["cbl", "gbl", "sbl"]:
        err = np.linalg.norm(krylov.apply(method, L, nodes, m, "exp", t=t).Y - ref)
        assert err <= bounds.lanczos_error_bound(len(nodes), m - 1, t, Lam) * (1 + 1e-9), method
    err = np.linalg.norm(krylov.apply("cheb", L, nodes, m, "exp", t=t).Y - ref)
    assert err <= bounds.cheb_error_bound(len(nodes), m, t, Lam) * (1 + 1e-9)


def test_lanczos_converges_faster_than_chebyshev():
    # Section 8.2: for equal m the classical block Lanczos error is the smallest
    g = synth.grid_graph((20, 20))
    L = _L(g)
    nodes = synth.sample_nodes(g.n, 8, seed=9)
    ref = dense.grid_exp_columns((20, 20), nodes, 2.0)
    e = {mth: _rel(krylov.apply(mth, L, nodes, 18, "exp", t=2.0).Y, ref)
         for mth in ["cbl", "gbl", "sbl", "cheb", "cheb2"]}
    assert all(e["cbl"] < e[k] for k in ["gbl", "sbl", "cheb", "cheb2"])
    assert max(e["gbl"], e["sbl"], e["cheb"]) < e["cheb2"]


def test_printed_constants_golden():
    vals = {}
    with open(os.path.join(GOLDEN, "stewart_leyk_constants.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    assert round(bounds.B_CONST, 3) == vals["b"]
    assert round(bounds.D_CONST, 3) == vals["d"]


# ------------------------------------------------------------------ planted mistakes
def _exactness_error(method="cbl"):
    g = synth.random_geometric_graph(300, 9, seed=15)
    L = _L(g)
    nodes = synth.sample_nodes(g.n, 5, seed=10)
    coeffs = [1.0, 0.3, 0.02, 0.001]
    r = krylov.apply(method, L, nodes, 5, "poly:" + ",".join(map(str, coeffs)))
    return _rel(r.Y, _poly_apply(L, nodes, coeffs))


def test_planted_transposed_offdiagonal_is_caught(monkeypatch):
    assert _exactness_error() < 1e-12
    monkeypatch.setattr(krylov, "_three_term", lambda L, Qk, Qp, Hpk: L @ Qk - Qp @ Hpk.T)
    assert _exactness_error() > 1e-6


def test_planted_dropped_three_term_is_caught(monkeypatch):
    monkeypatch.setattr(krylov, "_three_term", lambda L, Qk, Qp, Hpk: L @ Qk)
    assert _exactness_error() > 1e-6


def test_planted_wrong_sign_update_is_caught(monkeypatch):
    monkeypatch.setattr(krylov, "_subtract", lambda X, Qk, Hkk: X + Qk @ Hkk)
    assert _exactness_error() > 1e-6


def test_planted_unhalved_endpoint_is_caught(monkeypatch):
    m, Lam = 6, 10.0
    f = dense.phi_function("exp", t=0.3)
    monkeypatch.setattr(krylov, "cheb_series_weights", lambda mm: np.ones(mm + 1))
    c = krylov.cheb_coefficients(f, m, Lam)
    lam = krylov.lobatto_nodes(m, Lam)
    assert np.max(np.abs(krylov.cheb_eval_scalar(c, Lam, lam) - f(lam))) > 1e-6


def test_planted_transposed_eigvectors_is_caught(monkeypatch):
    g = synth.path_graph(9)
    f = dense.phi_function("exp", t=1.0)
    good = dense.kernel_columns(_Ld(g), [0, 3], f)
    real_eigh = np.linalg.eigh
    monkeypatch.setattr(np.linalg, "eigh", lambda A: (lambda w, V: (w, V.T))(*real_eigh(A)))
    bad = dense.kernel_columns(_Ld(g), [0, 3], f)
    ref = dense.path_function(9, f)[:, [0, 3]]
    assert np.max(np.abs(good - ref)) < 1e-12 and np.max(np.abs(bad - ref)) > 1e-6


# ----------------------------------------------------------------------------- RLS (Section 5)
from oracle import rls  # noqa: E402


def _rls_case(n=40, N=6, seed=20):
    # a connected graph (2-D grid with about n nodes), so that no Lanczos block breaks down
    side = int(round(np.sqrt(n)))
    g = synth.grid_graph((side, max(2, n // side)))
    L = krylov.laplacian(g.n, g.rowptr, g.col, g.val)
    nodes = synth.sample_nodes(g.n, N, seed=seed + 1)
    y = np.random.default_rng(seed).choice([-1.0, 1.0], size=N)
    return L, nodes, y


@pytest.mark.parametrize("phi,kw", [("exp", dict(t=2.0)), ("spline", dict(eps=0.1, s=2.0))])
def test_rls_gamma_zero_interpolates(phi, kw):
    # Section 2.3: with gamma = 0 the predictor interpolates the labels at W
    L, nodes, y = _rls_case()
    pred, c = rls.exact(L, nodes, y, 0.0, phi, **kw)
    assert np.allclose(pred[nodes], y, atol=1e-9)


def test_rls_residual_is_gamma_n_c():
    # (K + gamma N I) c = y  <=>  y - pred(W) = gamma N c; pins the gamma N scaling
    L, nodes, y = _rls_case()
    gamma = 0.3
    pred, c = rls.exact(L, nodes, y, gamma, "exp", t=1.0)
    assert np.allclose(y - pred[nodes], gamma * len(nodes) * c, atol=1e-12)
    # a planted mistake (gamma without the factor N) breaks the identity
    K = dense.kernel_columns(L.toarray(), nodes, dense.phi_function("exp", t=1.0))[nodes, :]
    c_bad = np.linalg.solve(K + gamma * np.eye(len(nodes)), y)
    assert not np.allclose(y - K @ c_bad, gamma * len(nodes) * c_bad, atol=1e-6)


def test_rls_krylov_exact_at_full_dimension():
    # m N >= n: the cbl columns are exact, so the Krylov predictor is the exact one
    L, nodes, y = _rls_case(n=30, N=6)
    pe, ce = rls.exact(L, nodes, y, 0.05, "spline", eps=0.1, s=1.0)
    pk, ck = rls.krylov_predictor("cbl", L, nodes, 6, y, 0.05, "spline", eps=0.1, s=1.0)
    assert np.allclose(pk, pe, rtol=1e-8, atol=1e-10)


def test_rls_algorithm3_equals_collocation_form():
    # Algorithm 3 (F_1^T phi(H_m) F_1, basis times phi(H_m) F_1 c) equals the general form
    # with E_W^T Y (identity from the proof of Theorem 3.1)
    L, nodes, y = _rls_case(n=60, N=5)
    p1, c1 = rls.cbl_alg3(L, nodes, 4, y, 0.01, "exp", t=1.5)
    p2, c2 = rls.krylov_predictor("cbl", L, nodes, 4, y, 0.01, "exp", t=1.5)
    assert np.allclose(c1, c2, rtol=1e-9, atol=1e-12)
    assert np.allclose(p1, p2, rtol=1e-9, atol=1e-12)


def test_rls_error_bound_of_section5():
    # the bound of Theorem 5.1 (first order): ||y - y_kr|| <= ||y|| / (phi_min + gamma N)
    # (1 + phi_max / (phi_min + gamma N)) ||phi(L) E_W - p(L) E_W||_2, checked with slack 2
    L, nodes, y = _rls_case(n=80, N=5, seed=23)
    gamma, t = 0.05, 1.0
    f = dense.phi_function("exp", t=t)
    lam = np.linalg.eigvalsh(L.toarray())
    pe, _ = rls.exact(L, nodes, y, gamma, "exp", t=t)
    Ye = dense.kernel_columns(L.toarray(), nodes, f)
    N = len(nodes)
    fmin, fmax = f(lam).min(), f(lam).max()
    for m in (3, 5, 8):
        pk, _ = rls.krylov_predictor("cbl", L, nodes, m, y, gamma, "exp", t=t)
        Yk = krylov.apply("cbl", L, nodes, m, "exp", t=t).Y
        bound = (np.linalg.norm(y) / (fmin + gamma * N) * (1 + fmax / (fmin + gamma * N))
                 * np.linalg.norm(Ye - Yk, 2))
        assert np.linalg.norm(pe - pk) <= 2 * bound + 1e-14


# ----------------------------------------------------------------------------- normalized L
@pytest.mark.parametrize("n", [5, 201])
def test_normalized_path_spectrum_closed_form(n):
    # the normalized Laplacian of the path P_n has eigenvalues 1 - cos(pi k / (n - 1))
    g = synth.path_graph(n)
    Ln = dense.normalized_laplacian_dense(_Ld(g))
    lam = np.sort(np.linalg.eigvalsh(Ln))
    ref = np.sort(1.0 - np.cos(np.pi * np.arange(n) / (n - 1)))
    assert np.allclose(lam, ref, atol=1e-12)


def test_normalized_laplacian_properties():
    # D^{1/2} 1 spans the kernel; spectrum in [0, 2]; isolated nodes give zero rows
    g = synth.random_geometric_graph(60, 5, seed=9)
    L = _Ld(g)
    Ln = dense.normalized_laplacian_dense(L)
    d = np.diag(L)
    assert np.allclose(Ln @ np.sqrt(d), 0.0, atol=1e-12)
    lam = np.linalg.eigvalsh(Ln)
    assert lam.min() > -1e-12 and lam.max() < 2 + 1e-12
    iso = np.where(d == 0)[0]
    assert np.all(Ln[iso, :] == 0.0)


def test_local_reorth_is_a_no_op_in_exact_arithmetic():
    # Q_k^T X = 0 and Q_{k-1}^T X = 0 in exact arithmetic, so the second local pass changes
    # the FP64 result only at rounding level while orthogonality holds
    g = synth.grid_graph((20, 20))
    L = _L(g)
    nodes = synth.sample_nodes(g.n, 5, seed=30)
    a = krylov.apply("cbl", L, nodes, 8, "exp", t=1.0).Y
    b = krylov.apply("cbl", L, nodes, 8, "exp", t=1.0, reorth="local").Y
    assert _rel(b, a) < 1e-12


# ----------------------------------------------------------------------------- full reorthogonalisation
# reorth=True is not in the paper: X -= Q_{1:k}(Q_{1:k}^T X), twice.  It is
# pinned by what it must achieve: it changes nothing in exact arithmetic (the Lanczos blocks
# are orthonormal, Theorem 3.1's setting), its output is the orthogonal projection of X onto
# the complement of the basis (orthogonal to the basis, and differing from X by an element of
# its span), and it keeps a long FP64 run orthonormal where the plain recurrence is not.
def _orth_defect(basis):
    B = np.hstack(basis)
    return float(np.linalg.norm(B.T @ B - np.eye(B.shape[1])))


def _projection_defects(seed=40, n=300, N=4, k=6, scale=1e-9):
    # X = B C + scale Z: almost inside the span of the basis, where one Gram-Schmidt pass
    # leaves a component of relative size u / scale along it
    rng = np.random.default_rng(seed)
    B, _ = np.linalg.qr(rng.standard_normal((n, k * N)))
    Q = [B[:, i * N:(i + 1) * N] for i in range(k)]
    X = B @ rng.standard_normal((k * N, N)) + scale * rng.standard_normal((n, N))
    out = krylov._reorthogonalise(X, Q)
    along = float(np.linalg.norm(B.T @ out) / np.linalg.norm(out))
    D = X - out
    coef = np.linalg.lstsq(B, D, rcond=None)[0]
    outside = float(np.linalg.norm(D - B @ coef) / np.linalg.norm(X))
    return along, outside


def _long_run_defects(m=40):
    # weighted Barabasi-Albert: a few hub eigenvalues converge within a few steps and the
    # FP64 three-term recurrence loses orthogonality (defect O(1) at m = 40)
    g = synth.barabasi_albert_graph(2000, 5, seed=3, weighted=True)
    L = _L(g)
    nodes = synth.sample_nodes(g.n, 2, seed=4)
    f = dense.phi_function("exp", t=1.0)
    plain = krylov.cbl(L, nodes, m, f)
    full = krylov.cbl(L, nodes, m, f, reorth=True)
    return _orth_defect(plain.basis), _orth_defect(full.basis)


def test_full_reorth_is_a_no_op_in_exact_arithmetic():
    g = synth.grid_graph((20, 20))
    L = _L(g)
    nodes = synth.sample_nodes(g.n, 5, seed=31)
    a = krylov.apply("cbl", L, nodes, 8, "exp", t=1.0)
    b = krylov.apply("cbl", L, nodes, 8, "exp", t=1.0, reorth=True)
    assert _rel(b.Y, a.Y) < 1e-12
    assert _orth_defect(a.basis) < 1e-13 and _orth_defect(b.basis) < 1e-13


def test_full_reorth_is_the_orthogonal_projection():
    along, outside = _projection_defects()
    assert along < 1e-12      # one pass: about 1e-7 here
    assert outside < 1e-13


def test_full_reorth_keeps_a_long_run_orthonormal():
    plain, full = _long_run_defects()
    assert plain > 1e-2       # the plain recurrence drifts (Paige)
    assert full < 1e-12


def _reorth_pins_hold():
    along, outside = _projection_defects()
    _, full = _long_run_defects()
    return along < 1e-12 and outside < 1e-13 and full < 1e-12


@pytest.mark.filterwarnings("ignore::RuntimeWarning")   # the flipped process overflows
def test_planted_reorth_sign_flip_is_caught(monkeypatch):
    def bad(X, Q):
        B = np.hstack(Q)
        for _ in range(2):
            X = X + B @ (B.T @ X)
        return X
    monkeypatch.setattr(krylov, "_reorthogonalise", bad)
    assert not _reorth_pins_hold()


def test_planted_reorth_single_pass_is_caught(monkeypatch):
    def bad(X, Q):
        B = np.hstack(Q)
        return X - B @ (B.T @ X)
    monkeypatch.setattr(krylov, "_reorthogonalise", bad)
    assert not _reorth_pins_hold()


def test_planted_reorth_without_newest_block_is_caught(monkeypatch):
    real = krylov._reorthogonalise
    monkeypatch.setattr(krylov, "_reorthogonalise", lambda X, Q: real(X, Q[:-1]) if len(Q) > 1 else X)
    assert not _reorth_pins_hold()
