"""The tensor-core (tcgen05, BF16 x 6 split products) kernels of the classical block Lanczos
step, through the C ABI with KB_TENSOR_CORES=1: parity with the FP64 oracle at the same
tolerance as the SIMT kernels, agreement with the SIMT path, and the frontier, two-pass and
reorthogonalisation paths on top of them.
"""
import numpy as np
import pytest

import synth
from test_gpu_parity import _oracle, _rel, tol32

pytestmark = pytest.mark.gpu


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
    return synth.random_geometric_graph(20000, 10, seed=1)


@pytest.fixture
def tc(monkeypatch):
    monkeypatch.setenv("KB_TENSOR_CORES", "1")


def _run(kb, G, phi, nodes, m, **kw):
    import torch
    Y, info = kb.kernel_columns(G, "cbl", phi, nodes, m, info=True, **kw)
    torch.cuda.synchronize()
    return Y.cpu().numpy().astype(np.float64), info


def _both(kb, g, phi, nodes, m, monkeypatch, **kw):
    with kb.Graph.from_csr(g) as G:
        monkeypatch.setenv("KB_TENSOR_CORES", "0")
        Ys, _ = _run(kb, G, phi, nodes, m, **kw)
        monkeypatch.setenv("KB_TENSOR_CORES", "1")
        Y, info = _run(kb, G, phi, nodes, m, **kw)
        lam = G.lambda_max
    assert info["status"] == 0
    ref = _oracle(g, "cbl", nodes, m, phi, **kw)
    return _rel(Y, ref), _rel(Ys, ref), lam


@pytest.mark.parametrize("t", [0.5, 2.0])
@pytest.mark.parametrize("M", [64, 48])
def test_tensor_core_cbl_exp_parity(kb, rgg, monkeypatch, t, M):
    # heat kernels: within the FP32 tolerance
    nodes = synth.sample_nodes(rgg.n, M, seed=11)
    err, err_simt, lam = _both(kb, rgg, "exp", nodes, 24, monkeypatch, t=t)
    print(f"tensor-core cbl exp t={t} M={M}: rel err {err:.2e} (SIMT {err_simt:.2e})")
    assert err < tol32("exp", lam, t=t)


def test_tensor_core_cbl_spline_error_ratio(kb, rgg, monkeypatch):
    # The tensor-core path is less accurate than the SIMT kernels on sensitive kernels: for
    # (0.1 I + L)^{-2} its error is 4-6x the SIMT error and about 1.5x the first-order FP32
    # bound, which is why it is not the default.  The SIMT result stays within the bound;
    # the tensor-core result is held to twice the bound.
    nodes = synth.sample_nodes(rgg.n, 64, seed=11)
    err, err_simt, lam = _both(kb, rgg, "spline", nodes, 24, monkeypatch, eps=0.1, s=2.0)
    bound = tol32("spline", lam, eps=0.1, s=2.0)
    print(f"tensor-core cbl spline eps=0.1 s=2: rel err {err:.2e} (SIMT {err_simt:.2e}, "
          f"FP32 bound {bound:.2e})")
    assert err_simt < bound
    assert err < 2 * bound


def test_tensor_core_agrees_with_simt(kb, rgg, monkeypatch):
    nodes = synth.sample_nodes(rgg.n, 64, seed=12)
    with kb.Graph.from_csr(rgg) as G:
        monkeypatch.setenv("KB_TENSOR_CORES", "0")
        Ys, _ = _run(kb, G, "exp", nodes, 30, t=1.0)
        monkeypatch.setenv("KB_TENSOR_CORES", "1")
        Yt, _ = _run(kb, G, "exp", nodes, 30, t=1.0)
    assert _rel(Yt, Ys) < 2 * tol32("exp", 1.0)


@pytest.mark.parametrize("nf", [0, 1])
def test_tensor_core_frontier_and_two_pass(kb, rgg, tc, nf):
    import torch
    nodes = synth.sample_nodes(rgg.n, 64, seed=13)
    with kb.Graph.from_csr(rgg) as G:
        Y1, i1 = kb.kernel_columns(G, "cbl", "exp", nodes, 20, info=True, t=2.0, no_frontier=nf)
        Y2, i2 = kb.kernel_columns(G, "cbl", "exp", nodes, 20, info=True, t=2.0, no_frontier=nf, two_pass=1)
        torch.cuda.synchronize()
    # the replay repeats the same tensor-core instructions on the same operands
    assert torch.equal(Y1, Y2)
    ref = _oracle(rgg, "cbl", nodes, 20, "exp", t=2.0)
    assert _rel(Y1.cpu().numpy().astype(np.float64), ref) < tol32("exp", 60.0, t=2.0)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_tensor_core_few_steps(kb, tc, m):
    g = synth.grid_graph((40, 40))
    nodes = synth.sample_nodes(g.n, 64, seed=14)
    with kb.Graph.from_csr(g) as G:
        Y, info = _run(kb, G, "exp", nodes, m, t=1.0)
    ref = _oracle(g, "cbl", nodes, m, "exp", t=1.0)
    assert _rel(Y, ref) < tol32("exp", 8.0)


def test_tensor_core_local_reorth_on_weighted_ba(kb, tc):
    ba = synth.barabasi_albert_graph(30_000, 5, seed=3, weighted=True)
    nodes = synth.sample_nodes(ba.n, 64, seed=4)
    with kb.Graph.from_csr(ba) as G:
        Y, info = _run(kb, G, "exp", nodes, 30, t=0.5, reorth=2)
        lam = G.lambda_max
    assert info["status"] == 0
    ref = _oracle(ba, "cbl", nodes, 30, "exp", t=0.5, reorth=2)
    err = _rel(Y, ref)
    print(f"tensor-core cbl local reorth, BA 3e4: rel err {err:.2e}")
    assert err < tol32("exp", lam, t=0.5)
