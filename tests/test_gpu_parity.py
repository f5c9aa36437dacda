"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: relative Frobenius error <= 1e-6 for the FP32 path and <= 1e-11 for the
plain FP64 mode (same arithmetic up to summation order).  Inputs are seeded synthetic
graphs shaped like the workloads: random geometric graphs of mean degree 10, 2-D grids,
weighted Barabasi-Albert graphs, path graphs.
"""
import numpy as np
import pytest

import synth
from oracle import dense, krylov

pytestmark = pytest.mark.gpu

TOL32 = 1e-6
METHODS = ["cbl", "gbl", "sbl", "cheb", "cheb2"]
U32 = 2.0 ** -24


def tol32(phi, lam, t=1.0, eps=0.01, s=1.0):
    """FP32-path tolerance: the 1e-6 bar, or, for kernels whose relative sensitivity to a
    perturbation of the spectrum exceeds it, the first-order bound kappa * Lambda * u32.
    Rounding the Krylov basis to FP32 perturbs the projected spectrum by O(u32 Lambda);
    |d log phi / d lambda| <= kappa with kappa = |t| for e^{-t lambda} and s/eps for
    (eps + lambda)^{-s}."""
    kappa = abs(t) if phi == "exp" else s / eps
    return max(TOL32, kappa * lam * U32)


@pytest.fixture(scope="module")
def kb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_06384_gb300 import kb as _kb
    import os
    if not os.path.exists(_kb.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _kb


def _gpu(kb, G, method, phi, nodes, m, info=False, **kw):
    import torch
    Y, r = kb.kernel_columns(G, method, phi, nodes, m, info=True, **kw)
    torch.cuda.synchronize()
    out = Y.cpu().numpy().astype(np.float64)
    return (out, r) if info else out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def check_err(label, err, bar):
    """Assert a measured relative error against its bar, printing both (lines starting with
    ERRLOG, collected by `pytest -s`, give the table of measured errors beside the 1e-6
    gate for every case that uses a conditioning-aware or BF16 bar)."""
    print(f"ERRLOG {label}: {err:.3e} (bar {bar:.2e})")
    assert err < bar, (label, err, bar)


def _oracle(g, method, nodes, m, phi, **kw):
    L = krylov.laplacian(g.n, g.rowptr, g.col, g.val)
    if kw.get("reorth") == 2:
        kw = dict(kw, reorth="local")
    return krylov.apply(method, L, nodes, m, phi, **kw).Y


@pytest.fixture(scope="module")
def rgg():
    return synth.random_geometric_graph(20000, 10, seed=1)


# ---------------------------------------------------------------- the small config
def test_grid_32x32_cbl_against_oracle_and_closed_form(kb):
    g = synth.grid_graph((32, 32))
    nodes = synth.sample_nodes(g.n, 16, seed=1)
    with kb.Graph.from_csr(g) as G:
        Y, info = _gpu(kb, G, "cbl", "exp", nodes, 20, info=True, t=1.0)
    ref = _oracle(g, "cbl", nodes, 20, "exp", t=1.0)
    assert _rel(Y, ref) < TOL32
    assert info["steps_done"] == 20 and info["spmm_launches"] == 20
    exact = dense.grid_exp_columns((32, 32), nodes, 1.0)
    assert _rel(Y, exact) < 1e-5   # approximation error of m = 20 (reported, loose)


# ---------------------------------------------------------------- all variants, RGG
@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("t", [0.5, 2.0])
def test_rgg_exp_parity(kb, rgg, method, t):
    nodes = synth.sample_nodes(rgg.n, 64, seed=2)
    with kb.Graph.from_csr(rgg) as G:
        Y, info = _gpu(kb, G, method, "exp", nodes, 30, info=True, t=t)
    ref = _oracle(rgg, method, nodes, 30, "exp", t=t)
    err = _rel(Y, ref)
    print(f"{method} t={t}: rel err {err:.3e}")
    assert err < TOL32
    assert info["spmm_launches"] == 30


@pytest.mark.parametrize("s", [2.0, 0.5, 1.5])
@pytest.mark.parametrize("method", METHODS)
def test_rgg_spline_parity(kb, rgg, method, s):
    # (eps I + L)^{-s} for every s > 0 (Section 2.4): integer s by floor(s) block solves of
    # the projected problem, the fractional rest of non-integer s by the quadrature over
    # real shifts; the oracle evaluates phi(H_m) by its eigendecomposition
    nodes = synth.sample_nodes(rgg.n, 32, seed=3)
    with kb.Graph.from_csr(rgg) as G:
        Y = _gpu(kb, G, method, "spline", nodes, 20, eps=0.1, s=s)
        Y64 = _gpu(kb, G, method, "spline", nodes, 20, eps=0.1, s=s, basis="f64")
        lam = G.lambda_max
    ref = _oracle(rgg, method, nodes, 20, "spline", eps=0.1, s=s)
    err, err64 = _rel(Y, ref), _rel(Y64, ref)
    check_err(f"rgg2e4 {method} spline eps=0.1 s={s:g} m=20 FP32", err, tol32("spline", lam, eps=0.1, s=s))
    check_err(f"rgg2e4 {method} spline eps=0.1 s={s:g} m=20 FP64", err64, 1e-7)


@pytest.mark.parametrize("method", ["cbl", "gbl", "sbl"])
@pytest.mark.parametrize("s", [0.3, 2.75])
def test_noninteger_spline_small_eps_weighted(kb, method, s):
    # a weighted hub-heavy graph with a small shift: (eps + Lambda) / eps ~ 1e5, where the
    # quadrature needs its most nodes.  The block process loses orthogonality on the hubs
    # even in FP64, so cbl runs (and is compared) with full reorthogonalisation
    g = synth.barabasi_albert_graph(3000, 5, seed=13, weighted=True)
    nodes = synth.sample_nodes(g.n, 12, seed=14)
    ro = 1 if method == "cbl" else 0
    with kb.Graph.from_csr(g) as G:
        Y64 = _gpu(kb, G, method, "spline", nodes, 14, eps=0.005, s=s, basis="f64", reorth=ro)
        Y = _gpu(kb, G, method, "spline", nodes, 14, eps=0.005, s=s, reorth=ro)
        lam = G.lambda_max
    ref = _oracle(g, method, nodes, 14, "spline", eps=0.005, s=s, reorth=bool(ro))
    check_err(f"ba3e3w {method} spline eps=0.005 s={s:g} m=14 FP64", _rel(Y64, ref), 1e-7)
    check_err(f"ba3e3w {method} spline eps=0.005 s={s:g} m=14 FP32", _rel(Y, ref), tol32("spline", lam, eps=0.005, s=s))


@pytest.mark.parametrize("method", ["cheb", "cheb2"])
def test_chebyshev_noninteger_spline(kb, rgg, method):
    nodes = synth.sample_nodes(rgg.n, 8, seed=4)
    with kb.Graph.from_csr(rgg) as G:
        Y = _gpu(kb, G, method, "spline", nodes, 24, eps=0.5, s=1.5)
    assert _rel(Y, _oracle(rgg, method, nodes, 24, "spline", eps=0.5, s=1.5)) < TOL32


# ---------------------------------------------------------------- widths and ragged cases
@pytest.mark.parametrize("M", [1, 5, 13, 33, 100, 128])
@pytest.mark.parametrize("method", METHODS)
def test_ragged_widths(kb, method, M):
    g = synth.random_geometric_graph(3001, 9, seed=5)
    nodes = synth.sample_nodes(g.n, M, seed=M)
    with kb.Graph.from_csr(g) as G:
        Y = _gpu(kb, G, method, "exp", nodes, 12, t=0.7)
    assert _rel(Y, _oracle(g, method, nodes, 12, "exp", t=0.7)) < TOL32


@pytest.mark.parametrize("method", ["sbl", "cheb", "cheb2"])
def test_wide_blocks_split_into_groups(kb, method):
    g = synth.random_geometric_graph(4000, 9, seed=6)
    nodes = synth.sample_nodes(g.n, 300, seed=7)
    with kb.Graph.from_csr(g) as G:
        Y = _gpu(kb, G, method, "exp", nodes, 10, t=1.0)
    assert _rel(Y, _oracle(g, method, nodes, 10, "exp", t=1.0)) < TOL32


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("method", METHODS)
def test_few_steps(kb, method, m):
    if method == "cheb2" and m < 2:
        pytest.skip("cheb2 needs m >= 2")
    g = synth.random_geometric_graph(2000, 9, seed=8)
    nodes = synth.sample_nodes(g.n, 10, seed=9)
    with kb.Graph.from_csr(g) as G:
        Y = _gpu(kb, G, method, "exp", nodes, m, t=1.3)
    assert _rel(Y, _oracle(g, method, nodes, m, "exp", t=1.3)) < TOL32


def test_weighted_generalized_laplacian(kb):
    # BA with float32 weights plus a positive diagonal excess: exercises the weight and
    # diagonal-excess loads of the SpMM
    g = synth.barabasi_albert_graph(3000, 5, seed=3, weighted=True)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    val = g.val.copy()
    diag = rows == g.col
    rng = np.random.default_rng(0)
    val[diag] = (val[diag] + rng.uniform(0, 0.5, size=g.n)).astype(np.float32)
    g2 = synth.CSRGraph(g.n, g.rowptr, g.col, val)
    nodes = synth.sample_nodes(g.n, 24, seed=11)
    with kb.Graph.from_csr(g2) as G:
        info = G.info()
        assert not info["standard_unit"]
        assert abs(info["lambda_max"] - krylov.gershgorin_bound(krylov.laplacian(g.n, g.rowptr, g.col, val))) < 1e-9 * info["lambda_max"]
        for method in METHODS:
            Y = _gpu(kb, G, method, "exp", nodes, 16, t=0.05)
            assert _rel(Y, _oracle(g2, method, nodes, 16, "exp", t=0.05)) < TOL32, method


def test_projected_bound_brackets_the_spectrum(kb):
    # the bound of the Lanczos projected series lies between lambda_max(L) (dense
    # eigenvalues) and the Gershgorin bound; for unit-weight D - A it is the edge bound
    # max (d_i + d_j) (Anderson and Morley), for a star graph exactly lambda_max = n
    n = 30
    star = synth.from_edges(n, np.zeros(n - 1, dtype=np.int64), np.arange(1, n))
    cases = [star, synth.barabasi_albert_graph(400, 3, seed=2),
             synth.barabasi_albert_graph(400, 3, seed=2, weighted=True), synth.grid_graph((9, 7))]
    for g in cases:
        lmax = np.linalg.eigvalsh(dense.laplacian_dense(g.n, g.rowptr, g.col, g.val)).max()
        with kb.Graph.from_csr(g) as G:
            info = G.info()
        assert lmax <= info["lambda_projected"] * (1 + 1e-12)
        assert info["lambda_projected"] <= info["lambda_max"] * (1 + 1e-12)
        if info["standard_unit"]:
            rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
            off = rows != g.col
            deg = np.bincount(rows[off], minlength=g.n)
            edge = (deg[rows[off]] + deg[g.col[off]]).max()
            assert abs(info["lambda_projected"] - min(info["lambda_max"], edge * 1.001)) < 1e-9 * edge
    # the star: the bound is tight up to its margin of 1e-3
    with kb.Graph.from_csr(star) as G:
        assert abs(G.info()["lambda_projected"] - n * 1.001) < 1e-9


@pytest.mark.parametrize("t", [0.05, 0.5, 3.0])
def test_star_graph_exp_lanczos_with_tight_bound(kb, t):
    # (t = 3: t Lambda = 6e3, a series of thousands of terms, which the tridiagonal step of
    # gbl / sbl applies in chunks)
    # the edge bound meets lambda_max exactly on a star: the projected series must still
    # cover the Ritz values the FP32 process produces
    n = 2001
    g = synth.from_edges(n, np.zeros(n - 1, dtype=np.int64), np.arange(1, n))
    with kb.Graph.from_csr(g) as G:
        for method in ("cbl", "gbl", "sbl"):
            # (several leaves in one cbl block give a rank-deficient block: centre only)
            nodes = [0] if method == "cbl" else [0, 5, 17, 900]
            Y = _gpu(kb, G, method, "exp", nodes, 6, t=t)
            lam = G.lambda_max
            check_err(f"star2001 {method} exp t={t} m=6 FP32", _rel(Y, _oracle(g, method, nodes, 6, "exp", t=t)),
                      tol32("exp", lam, t=t))


# ---------------------------------------------------------------- exactness and stops
def test_cbl_exact_at_full_dimension(kb):
    g = synth.random_weighted_graph(12, 0.5, seed=7)
    nodes = [0, 5, 9]
    with kb.Graph.from_csr(g) as G:
        Y = _gpu(kb, G, "cbl", "exp", nodes, 4, t=0.8)
    exact = dense.kernel_columns(dense.laplacian_dense(g.n, g.rowptr, g.col, g.val), nodes,
                                 dense.phi_function("exp", t=0.8))
    assert _rel(Y, exact) < TOL32


def test_invariant_subspace_stops_early(kb):
    g = synth.from_edges(6, np.array([0, 1, 3]), np.array([1, 2, 4]))
    nodes = [0, 1, 2]
    exact = dense.kernel_columns(dense.laplacian_dense(g.n, g.rowptr, g.col, g.val), nodes,
                                 dense.phi_function("exp", t=1.0))
    with kb.Graph.from_csr(g) as G:
        Y, info = _gpu(kb, G, "cbl", "exp", nodes, 5, info=True, t=1.0)
        assert info["steps_done"] == 1
        assert _rel(Y, exact) < TOL32
        Y, info = _gpu(kb, G, "gbl", "exp", nodes, 5, info=True, t=1.0)
        assert _rel(Y, _oracle(g, "gbl", nodes, 5, "exp", t=1.0)) < TOL32


def test_breakdown_is_reported(kb):
    # path 0-1-2 with W = {0, 2}: X = [-e_1, -e_1] after the projection is rank one
    g = synth.path_graph(3)
    with kb.Graph.from_csr(g) as G:
        with pytest.raises(kb.KbError) as ei:
            _gpu(kb, G, "cbl", "exp", [0, 2], 3, t=1.0)
    assert ei.value.code == -6
    with pytest.raises(krylov.Breakdown):
        _oracle(g, "cbl", [0, 2], 3, "exp", t=1.0)


@pytest.mark.parametrize("M", [4, 16, 64])
def test_breakdown_at_a_middle_pivot(kb, M):
    # an isolated node in the second column of the block: L e_w = 0, so column 1 of the new
    # block X is exactly zero while the others are not; the Cholesky factorisation of X^T X
    # meets a zero pivot at index 1 <= M - 2, found by the look-ahead warp while the other
    # warps still update the trailing rows
    b = synth.random_geometric_graph(3001, 9, seed=5)   # the graph of test_ragged_widths
    rows = np.repeat(np.arange(b.n), np.diff(b.rowptr))
    up = rows < b.col
    n = b.n + 1                                          # node n - 1 has no edges
    g = synth.from_edges(n, rows[up], b.col[up])
    nodes = [int(x) for x in synth.sample_nodes(b.n, M, seed=M)]
    nodes[1] = n - 1
    with kb.Graph.from_csr(g) as G:
        for _ in range(2):   # the same status twice: the context survives the breakdown
            with pytest.raises(kb.KbError) as ei:
                _gpu(kb, G, "cbl", "exp", nodes, 6, t=1.0)
            assert ei.value.code == -6
        # a node set without the isolated node still runs
        ok = [x for x in nodes if x != n - 1][: M - 1]
        Y = _gpu(kb, G, "cbl", "exp", ok, 6, t=1.0)
    assert _rel(Y, _oracle(g, "cbl", ok, 6, "exp", t=1.0)) < TOL32
    with pytest.raises(krylov.Breakdown):
        _oracle(g, "cbl", nodes, 6, "exp", t=1.0)


def test_path_single_column_all_lanczos_agree(kb):
    # the path graph of the paper's first experiment (n = 201, centre node), standard
    # Laplacian, e^{-20 L}
    n = 201
    g = synth.path_graph(n)
    with kb.Graph.from_csr(g) as G:
        lam = G.lambda_max
        outs = [_gpu(kb, G, mth, "exp", [100], 40, t=20.0) for mth in ["cbl", "gbl", "sbl"]]
        outs64 = [_gpu(kb, G, mth, "exp", [100], 40, t=20.0, basis="f64") for mth in ["cbl", "gbl", "sbl"]]
    ref = _oracle(g, "cbl", [100], 40, "exp", t=20.0)
    for mth, Y, Y64 in zip(["cbl", "gbl", "sbl"], outs, outs64):
        check_err(f"path201 {mth} exp t=20 m=40 FP32", _rel(Y, ref), tol32("exp", lam, t=20.0))
        assert _rel(Y64, ref) < 1e-7


# ---------------------------------------------------------------- frontier restriction
@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("M", [5, 16, 64, 128])
def test_frontier_restriction_matches_full_rows(kb, method, M):
    # the per-step kernels touch only rows within k hops of W; the skipped rows are exact
    # zeros, so the result equals the all-rows run up to summation order
    g = synth.random_geometric_graph(30000, 10, seed=41)
    nodes = synth.sample_nodes(g.n, M, seed=42)
    with kb.Graph.from_csr(g) as G:
        Yf = _gpu(kb, G, method, "exp", nodes, 20, t=1.0)
        Ya = _gpu(kb, G, method, "exp", nodes, 20, t=1.0, no_frontier=1)
    assert _rel(Yf, Ya) < 1e-6
    if method in ("cheb", "cheb2"):
        assert np.array_equal(Yf, Ya)   # same kernels, same row arithmetic
    assert _rel(Yf, _oracle(g, method, nodes, 20, "exp", t=1.0)) < TOL32


def test_frontier_unreached_rows_are_zero(kb):
    # two components; nodes in one: rows of the other component are never reached
    g1 = synth.random_geometric_graph(5000, 10, seed=43)
    g2 = synth.random_geometric_graph(5000, 10, seed=44)
    r1, c1 = np.repeat(np.arange(5000), np.diff(g1.rowptr)), g1.col
    r2, c2 = np.repeat(np.arange(5000), np.diff(g2.rowptr)), g2.col
    m1, m2 = r1 < c1, r2 < c2
    g = synth.from_edges(10000, np.concatenate([r1[m1], r2[m2] + 5000]),
                         np.concatenate([c1[m1], c2[m2] + 5000]))
    nodes = synth.sample_nodes(5000, 12, seed=45)
    for method in METHODS:
        with kb.Graph.from_csr(g) as G:
            Y = _gpu(kb, G, method, "exp", nodes, 15, t=0.5)
        assert np.all(Y[5000:] == 0.0), method
        assert _rel(Y, _oracle(g, method, nodes, 15, "exp", t=0.5)) < TOL32, method


def test_frontier_with_reorth_and_spline(kb):
    g = synth.barabasi_albert_graph(6000, 3, seed=46, weighted=True)
    nodes = synth.sample_nodes(g.n, 16, seed=47)
    with kb.Graph.from_csr(g) as G:
        lam = G.lambda_max
        Yf = _gpu(kb, G, "cbl", "spline", nodes, 10, eps=0.5, s=2.0, reorth=1)
        Ya = _gpu(kb, G, "cbl", "spline", nodes, 10, eps=0.5, s=2.0, reorth=1, no_frontier=1)
    ref = krylov.apply("cbl", krylov.laplacian(g.n, g.rowptr, g.col, g.val), nodes, 10,
                       "spline", eps=0.5, s=2.0, reorth=True).Y
    assert _rel(Yf, Ya) < 1e-6
    check_err("ba6e3w cbl spline eps=0.5 s=2 m=10 reorth=1 FP32", _rel(Yf, ref), tol32("spline", lam, eps=0.5, s=2.0))


# ---------------------------------------------------------------- full reorthogonalisation
@pytest.mark.parametrize("phi,kw", [("exp", dict(t=1.0)), ("spline", dict(eps=0.5, s=2.0))])
@pytest.mark.parametrize("M", [8, 64])
def test_cbl_full_reorthogonalisation_parity(kb, phi, kw, M):
    g = synth.barabasi_albert_graph(4000, 5, seed=31, weighted=True)
    nodes = synth.sample_nodes(g.n, M, seed=32)
    L = krylov.laplacian(g.n, g.rowptr, g.col, g.val)
    ref = krylov.apply("cbl", L, nodes, 12, phi, reorth=True, **kw).Y
    with kb.Graph.from_csr(g) as G:
        lam = G.lambda_max
        Y = _gpu(kb, G, "cbl", phi, nodes, 12, reorth=1, **kw)
        Y64 = _gpu(kb, G, "cbl", phi, nodes, 12, reorth=1, basis="f64", **kw)
    check_err(f"ba4e3w cbl {phi} {kw} M={M} m=12 reorth=1 FP32", _rel(Y, ref), tol32(phi, lam, **kw))
    assert _rel(Y64, ref) < 1e-7


def test_reorthogonalisation_keeps_long_runs_accurate(kb):
    # a long run on a small graph: loss of orthogonality in FP32 without reorthogonalisation,
    # agreement with the reorthogonalised FP64 oracle with it
    g = synth.random_geometric_graph(600, 8, seed=33)
    nodes = synth.sample_nodes(g.n, 4, seed=34)
    L = krylov.laplacian(g.n, g.rowptr, g.col, g.val)
    ref = krylov.apply("cbl", L, nodes, 40, "exp", t=0.5, reorth=True).Y
    with kb.Graph.from_csr(g) as G:
        Yr = _gpu(kb, G, "cbl", "exp", nodes, 40, t=0.5, reorth=1)
    assert _rel(Yr, ref) < TOL32


def test_reorth_rejected_for_other_methods(kb):
    import torch
    g = synth.path_graph(40)
    with kb.Graph.from_csr(g) as G:
        Y = torch.empty((40, 2), dtype=torch.float32, device="cuda")
        with pytest.raises(kb.KbError) as ei:
            kb.kb_krylov_apply(G, "gbl", "exp", kb.make_params(t=1.0, reorth=1), np.array([3, 9]), 2, 5, Y)
        assert ei.value.code == -7


# ---------------------------------------------------------------- plain FP64 mode
@pytest.mark.parametrize("method", METHODS)
def test_fp64_mode_parity(kb, method):
    g = synth.random_geometric_graph(5000, 10, seed=12)
    nodes = synth.sample_nodes(g.n, 16, seed=13)
    with kb.Graph.from_csr(g) as G:
        Y = _gpu(kb, G, method, "exp", nodes, 20, t=2.0, basis="f64")
    # the result is returned in FP32, so FP32 output rounding bounds the agreement
    assert _rel(Y, _oracle(g, method, nodes, 20, "exp", t=2.0)) < 1e-7


@pytest.mark.parametrize("method", METHODS)
def test_fp64_mode_tight(kb, method):
    # FP64 throughout: agreement far below the FP32 tolerance (result stored as FP32, so
    # the comparison is against the FP32 rounding of the oracle)
    g = synth.random_geometric_graph(2000, 10, seed=14)
    nodes = synth.sample_nodes(g.n, 8, seed=15)
    with kb.Graph.from_csr(g) as G:
        Y = _gpu(kb, G, method, "exp", nodes, 15, t=1.0, basis="f64")
    ref = _oracle(g, method, nodes, 15, "exp", t=1.0)
    ref32 = ref.astype(np.float32).astype(np.float64)
    assert _rel(Y, ref32) < 1e-8


# ---------------------------------------------------------------- BF16 basis mode
U_BF16 = 2.0 ** -9


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("t", [0.5, 2.0])
def test_bf16_basis_parity(kb, rgg, method, t):
    # blocks stored in BF16 (unit roundoff u = 2^-9), arithmetic in FP32.  Every stored
    # element carries a relative rounding error up to u (about u/sqrt(3) r.m.s.), so the
    # assembled result cannot be closer than about 1e-3; the recurrences amplify the
    # rounding by the conditioning of the polynomial (measured 1.5e-3 to 1.9e-2 on these
    # cases), and the bar is 16 u = 3.1e-2
    nodes = synth.sample_nodes(rgg.n, 64, seed=2)
    with kb.Graph.from_csr(rgg) as G:
        Y, info = _gpu(kb, G, method, "exp", nodes, 30, info=True, t=t, basis="bf16")
    ref = _oracle(rgg, method, nodes, 30, "exp", t=t)
    err = _rel(Y, ref)
    print(f"ERRLOG rgg2e4 {method} exp t={t} m=30 BF16 basis: {err:.3e} (bar {16 * U_BF16:.2e})")
    assert np.isfinite(Y).all()
    assert err < 16 * U_BF16
    assert info["spmm_launches"] == 30


@pytest.mark.parametrize("method", METHODS)
def test_bf16_basis_spline_and_ragged(kb, method):
    g = synth.random_geometric_graph(6000, 10, seed=21)
    nodes = synth.sample_nodes(g.n, 37, seed=22)
    with kb.Graph.from_csr(g) as G:
        Y = _gpu(kb, G, method, "spline", nodes, 16, eps=0.5, s=2.0, basis="bf16")
    ref = _oracle(g, method, nodes, 16, "spline", eps=0.5, s=2.0)
    err = _rel(Y, ref)
    print(f"ERRLOG bf16 spline {method}: {err:.3e} (bar {16 * U_BF16:.2e})")
    assert err < 16 * U_BF16


# ---------------------------------------------------------------- entry points and errors
def test_host_output_matches_device_output(kb, rgg):
    import torch
    nodes = synth.sample_nodes(rgg.n, 20, seed=16)
    with kb.Graph.from_csr(rgg) as G:
        for method in METHODS:
            Yd = _gpu(kb, G, method, "exp", nodes, 10, t=1.0)
            Yh = torch.empty((rgg.n, 20), dtype=torch.float32).pin_memory()
            kb.kb_krylov_apply_host(G, method, "exp", kb.make_params(t=1.0), nodes, 20, 10, Yh)
            assert np.array_equal(Yh.numpy().astype(np.float64), Yd), method
            Yn = np.empty((rgg.n, 20), dtype=np.float32)   # pageable host memory
            kb.kb_krylov_apply_host(G, method, "exp", kb.make_params(t=1.0), nodes, 20, 10, Yn)
            assert np.array_equal(Yn.astype(np.float64), Yd), method


def test_argument_errors(kb):
    import torch
    g = synth.path_graph(50)
    with kb.Graph.from_csr(g) as G:
        Y = torch.empty((50, 4), dtype=torch.float32, device="cuda")
        p = kb.make_params(t=1.0)
        cases = [
            (dict(nodes=[1, 2, 2, 3], M=4, m=5, method="cbl"), -3),
            (dict(nodes=[1, 2, 3, 60], M=4, m=5, method="cbl"), -3),
            (dict(nodes=[1, 2, 3, 4], M=4, m=0, method="cbl"), -1),
            (dict(nodes=[1, 2, 3, 4], M=4, m=1, method="cheb2"), -1),
        ]
        for kw, code in cases:
            with pytest.raises(kb.KbError) as ei:
                kb.kb_krylov_apply(G, kw["method"], "exp", p, np.array(kw["nodes"]), kw["M"], kw["m"], Y)
            assert ei.value.code == code, (kw, str(ei.value))
        # non-integer s is supported (quadrature of the fractional power); s >= 65 is not
        kb.kb_krylov_apply(G, "cbl", "spline", kb.make_params(eps=0.1, s=1.5), np.arange(4), 4, 5, Y)
        with pytest.raises(kb.KbError) as ei:
            kb.kb_krylov_apply(G, "cbl", "spline", kb.make_params(eps=0.1, s=65.5), np.arange(4), 4, 5, Y)
        assert ei.value.code == -7
        with pytest.raises(kb.KbError) as ei:
            kb.kb_krylov_apply(G, "cbl", "exp", kb.make_params(t=1.0, basis=7), np.arange(4), 4, 5, Y)
        assert ei.value.code == -1


def test_stream_ordering_and_no_sync_without_info(kb, rgg):
    import torch
    nodes = synth.sample_nodes(rgg.n, 16, seed=17)
    s = torch.cuda.Stream()
    with kb.Graph.from_csr(rgg) as G:
        ref = _gpu(kb, G, "cbl", "exp", nodes, 12, t=1.0)
        with torch.cuda.stream(s):
            Y = torch.empty((rgg.n, 16), dtype=torch.float32, device="cuda")
            kb.kb_krylov_apply(G, "cbl", "exp", kb.make_params(t=1.0), nodes, 16, 12, Y, stream=s)
        s.synchronize()
        assert np.array_equal(Y.cpu().numpy().astype(np.float64), ref)


# ---------------------------------------------------------------- loss of orthogonality
@pytest.fixture(scope="module")
def ba():
    return synth.barabasi_albert_graph(50_000, 5, seed=3, weighted=True)


def test_lost_orthogonality_is_reported_not_returned(kb, ba):
    # weighted BA graph: the hub eigenvalues converge within a few steps and the FP32 block
    # Lanczos basis (reorth = 0) loses orthogonality (the FP64 process keeps the projected
    # spectrum in [0, Lambda], the FP32 one may not).  The call either reports
    # KB_ERR_ORTHOGONALITY (Y = NaN) or returns values within the bound max phi on
    # [0, Lambda]; accuracy on such graphs needs reorth = 2 (next test).
    nodes = synth.sample_nodes(ba.n, 64, seed=4)
    with kb.Graph.from_csr(ba) as G:
        for phi, kw, bound in (("exp", dict(t=0.5), 1.25), ("spline", dict(eps=1.0, s=2.0), 1.25)):
            try:
                Y, info = _gpu(kb, G, "cbl", phi, nodes, 30, info=True, **kw)
            except kb.KbError as e:
                assert e.code == -9
                continue
            assert np.isfinite(Y).all() and np.abs(Y).max() <= bound
            ref = _oracle(ba, "cbl", nodes, 30, phi, **kw)
            print(f"BA 5e4 cbl {phi} reorth=0: rel err {_rel(Y, ref):.2e} (no error reported)")


@pytest.mark.parametrize("phi,kw", [("exp", dict(t=0.5)), ("spline", dict(eps=1.0, s=2.0))])
def test_local_reorth_keeps_fp32_on_the_oracle(kb, ba, phi, kw):
    # reorth = 2 (second Gram-Schmidt pass against Q_k, Q_{k-1}) keeps the FP32 process on
    # the FP64 one on the same BA graph
    nodes = synth.sample_nodes(ba.n, 64, seed=4)
    with kb.Graph.from_csr(ba) as G:
        Y, info = _gpu(kb, G, "cbl", phi, nodes, 30, info=True, reorth=2, **kw)
        lam = G.lambda_max
    ref = _oracle(ba, "cbl", nodes, 30, phi, reorth=2, **kw)
    err = _rel(Y, ref)
    assert info["status"] == 0
    check_err(f"ba5e4w cbl {phi} {kw} M=64 m=30 reorth=2 FP32", err, tol32(phi, lam, **kw))


# ---------------------------------------------------------------- two-pass Lanczos
@pytest.mark.parametrize("method,kw", [("gbl", {}), ("sbl", {}), ("cbl", {}), ("cbl", dict(reorth=2))])
@pytest.mark.parametrize("nf", [0, 1])
def test_two_pass_reproduces_the_stored_basis_result(kb, rgg, method, kw, nf):
    # the second pass repeats the products and updates with the recorded coefficients, so
    # the blocks are bit-identical, and the accumulator of Y continues from the stored
    # partial sums: the result equals the one-pass result exactly
    import torch
    nodes = synth.sample_nodes(rgg.n, 48, seed=8)
    with kb.Graph.from_csr(rgg) as G:
        Y1, i1 = kb.kernel_columns(G, method, "exp", nodes, 24, info=True, t=2.0, no_frontier=nf, **kw)
        Y2, i2 = kb.kernel_columns(G, method, "exp", nodes, 24, info=True, t=2.0, no_frontier=nf,
                                   two_pass=1, **kw)
        torch.cuda.synchronize()
        p1 = kb.make_params(t=2.0, no_frontier=nf, **kw)
        p2 = kb.make_params(t=2.0, no_frontier=nf, two_pass=1, **kw)
        w1 = [kb.kb_workspace_bytes(G, method, "exp", p1, 48, m) for m in (24, 48)]
        w2 = [kb.kb_workspace_bytes(G, method, "exp", p2, 48, m) for m in (24, 48)]
    assert i2["spmm_launches"] == 2 * 24 - 1
    assert torch.equal(Y1, Y2), float((Y1 - Y2).abs().max())
    # scratch: a few n x W blocks instead of m of them; what still grows with m are the
    # per-step W x W coefficient records, far less than one stored block per step
    assert w2[0] < 0.3 * w1[0]
    assert (w2[1] - w2[0]) < 0.2 * (w1[1] - w1[0])


def test_two_pass_spline_and_errors(kb, rgg):
    import torch
    nodes = synth.sample_nodes(rgg.n, 16, seed=9)
    with kb.Graph.from_csr(rgg) as G:
        Y = _gpu(kb, G, "cbl", "spline", nodes, 16, eps=0.1, s=2.0, two_pass=1)
        lam = G.lambda_max
        Yr = torch.empty((rgg.n, 16), dtype=torch.float32, device="cuda")
        with pytest.raises(kb.KbError) as ei:
            kb.kb_krylov_apply(G, "cbl", "exp", kb.make_params(t=1.0, reorth=1, two_pass=1),
                               nodes, 16, 8, Yr)
        assert ei.value.code == -7
    ref = _oracle(rgg, "cbl", nodes, 16, "spline", eps=0.1, s=2.0)
    check_err("rgg2e4 cbl spline eps=0.1 s=2 m=16 two-pass FP32", _rel(Y, ref), tol32("spline", lam, eps=0.1, s=2.0))
