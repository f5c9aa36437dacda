"""The stopping rule of the serving workload for cbl (params.tol > 0), through the C ABI:
the process stops at the first check step k with ||U_k - [U_k'; 0]||_F <= tol ||U_k||_F, and
the result is exactly that of the fixed-m call with m = k.
"""
import numpy as np
import pytest

import synth
from test_gpu_parity import _oracle, _rel, tol32

pytestmark = pytest.mark.gpu

CHECKS = (8, 12, 16, 24, 32, 48, 64, 96)


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


@pytest.mark.parametrize("phi,kw", [("exp", dict(t=0.5)), ("exp", dict(t=3.0)),
                                    ("spline", dict(eps=0.5, s=2.0)), ("spline", dict(eps=0.5, s=1.5))])
def test_stopping_rule_matches_fixed_m(kb, rgg, phi, kw):
    import torch
    nodes = synth.sample_nodes(rgg.n, 32, seed=21)
    with kb.Graph.from_csr(rgg) as G:
        Ya, ia = kb.kernel_columns(G, "cbl", phi, nodes, 100, info=True, tol=1e-6, **kw)
        k = ia["steps_done"]
        Yf, fi = kb.kernel_columns(G, "cbl", phi, nodes, k, info=True, **kw)
        torch.cuda.synchronize()
        lam = G.lambda_max
    print(f"stopping rule {phi} {kw}: stopped after {k} steps")
    assert k in CHECKS
    assert fi["steps_done"] == k
    assert torch.equal(Ya, Yf)
    # the estimate that stopped the process is reported; the fixed-m call ran no check
    assert 0.0 <= ia["est_change"] <= 1e-6
    assert fi["est_change"] == -1.0
    Y = Ya.cpu().numpy().astype(np.float64)
    assert _rel(Y, _oracle(rgg, "cbl", nodes, k, phi, **kw)) < tol32(phi, lam, **kw)
    # the stopped result is within a small multiple of tol of the converged one
    ref = _oracle(rgg, "cbl", nodes, 64, phi, **kw)
    assert _rel(Y, ref) < 2e-5


def test_stopping_rule_errors(kb, rgg):
    import torch
    nodes = synth.sample_nodes(rgg.n, 8, seed=22)
    Y = torch.empty((rgg.n, 8), dtype=torch.float32, device="cuda")
    with kb.Graph.from_csr(rgg) as G:
        for method, p, code in (("gbl", kb.make_params(t=1.0, tol=1e-6), -7),
                                ("cbl", kb.make_params(t=1.0, tol=1e-6, two_pass=1), -7),
                                ("cbl", kb.make_params(t=1.0, tol=-1.0), -1)):
            with pytest.raises(kb.KbError) as ei:
                kb.kb_krylov_apply(G, method, "exp", p, nodes, 8, 20, Y)
            assert ei.value.code == code
        # a tolerance no check meets: all m steps run
        Y2, info = kb.kernel_columns(G, "cbl", "exp", nodes, 20, info=True, t=1.0, tol=1e-30)
        assert info["steps_done"] == 20
        # checks ran at steps 8, 12 and 16: the last one compared 16 with 12
        assert 1e-30 < info["est_change"] < 1.0
