"""RLS predictor (Section 5, Algorithm 3) through kb_rls_predict against the FP64 oracle.

The predictor inherits the kernel-column error amplified by the conditioning of the
collocation system: with relative column error d (the FP32 bar of the columns: 1e-6, or
kappa_phi Lambda u32 for kernels more sensitive than that), the coefficients move by about
kappa(E_W^T Y + gamma N I) d, so the bar is (1 + kappa) d.
"""
import numpy as np
import pytest

import synth
from oracle import krylov, rls

pytestmark = pytest.mark.gpu

METHODS = ["cbl", "gbl", "sbl", "cheb", "cheb2"]


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


@pytest.fixture(scope="module")
def rgg():
    return synth.random_geometric_graph(20000, 10, seed=51)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("phi,kw,gamma", [("exp", dict(t=1.0), 1e-3), ("spline", dict(eps=0.1, s=2.0), 1e-2)])
def test_rls_predictor_parity(kb, rgg, method, phi, kw, gamma):
    import torch
    nodes = synth.sample_nodes(rgg.n, 40, seed=52)
    y = np.random.default_rng(53).choice([-1.0, 1.0], size=nodes.size)
    L = krylov.laplacian(rgg.n, rgg.rowptr, rgg.col, rgg.val)
    ref, cref = rls.krylov_predictor(method, L, nodes, 24, y, gamma, phi, **kw)
    Yo = krylov.apply(method, L, nodes, 24, phi, **kw).Y
    kappa = np.linalg.cond(Yo[nodes, :] + gamma * nodes.size * np.eye(nodes.size))
    with kb.Graph.from_csr(rgg) as G:
        out = torch.empty(rgg.n, dtype=torch.float32, device="cuda")
        c = kb.kb_rls_predict(G, method, phi, kb.make_params(**kw), nodes, 24, y, gamma, out)
        pred = out.cpu().numpy().astype(np.float64)
        lam = G.lambda_max
    err = np.linalg.norm(pred - ref) / np.linalg.norm(ref)
    errc = np.linalg.norm(c - cref) / np.linalg.norm(cref)
    sens = kw["t"] if phi == "exp" else kw["s"] / kw["eps"]
    d = max(1e-6, sens * lam * 2.0 ** -24)
    print(f"rls {method} {phi}: kappa {kappa:.1e}, predictor rel err {err:.2e}, c rel err {errc:.2e}")
    assert err < (1 + kappa) * d
    assert errc < (1 + kappa) * d


def test_rls_interpolates_with_gamma_zero(kb):
    # gamma = 0: y_pred(W) = E_W^T Y c = y for any m (the collocation system itself)
    g = synth.grid_graph((12, 12))
    nodes = synth.sample_nodes(g.n, 16, seed=54)
    y = np.random.default_rng(55).standard_normal(nodes.size)
    import torch
    with kb.Graph.from_csr(g) as G:
        out = torch.empty(g.n, dtype=torch.float32, device="cuda")
        kb.kb_rls_predict(G, "cbl", "spline", kb.make_params(eps=0.5, s=1.0), nodes, 6, y, 0.0, out)
        pred = out.cpu().numpy().astype(np.float64)
    assert np.allclose(pred[nodes.astype(np.int64)], y, rtol=1e-4, atol=1e-4)


def test_rls_argument_errors(kb):
    import torch
    g = synth.grid_graph((8, 8))
    with kb.Graph.from_csr(g) as G:
        out = torch.empty(g.n, dtype=torch.float32, device="cuda")
        with pytest.raises(kb.KbError) as ei:
            kb.kb_rls_predict(G, "cbl", "exp", kb.make_params(t=1.0), np.arange(4), 5, np.ones(4), -1.0, out)
        assert ei.value.code == -1
        with pytest.raises(kb.KbError) as ei:
            kb.kb_rls_predict(G, "cbl", "exp", kb.make_params(t=1.0), np.array([1, 1]), 5, np.ones(2), 0.1, out)
        assert ei.value.code == -3
