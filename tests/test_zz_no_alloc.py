"""kb_cheb_apply_fixed_scratch: the Chebyshev solve for callers that cannot allocate.

Some callers cannot allocate device memory when they need kernel columns (a framework
that owns all device memory through its own allocator, a latency-critical loop that must
not enter an allocator, a process under a fixed memory budget).  The library gives them
one entry point whose scratch is a fixed device array inside the library.  These tests
call it through the C ABI and compare it with kb_krylov_apply(KB_CHEB) on the same
inputs, twice in a row (the second call reuses the scratch the first one left behind):
the two entry points run the same SpMM kernel with the same coefficients on every row
that is not exactly zero, so the results must be bitwise equal; both are also compared
element by element with the FP64 oracle.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth
from oracle import krylov

pytestmark = pytest.mark.gpu

TOL32 = 1e-6


@pytest.fixture(scope="module")
def kb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_2301_06384_gb300 import kb as _kb
    if not os.path.exists(_kb.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _kb


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("phi,kw", [("exp", dict(t=2.0)), ("spline", dict(eps=0.5, s=1.5))])
def test_fixed_scratch_matches_allocating_entry_point(kb, phi, kw):
    import torch
    g = synth.random_geometric_graph(20000, 10, seed=21)
    nodes = synth.sample_nodes(g.n, 64, seed=22)
    p = kb.make_params(**kw)
    with kb.Graph.from_csr(g) as G:
        ref = torch.empty((g.n, 64), dtype=torch.float32, device="cuda")
        kb.kb_krylov_apply(G, "cheb", phi, p, nodes, 64, 30, ref)
        torch.cuda.synchronize()
        refh = ref.cpu().numpy().astype(np.float64)
        for _ in range(2):
            Y = torch.full((g.n, 64), float("nan"), dtype=torch.float32, device="cuda")
            kb.kb_cheb_apply_fixed_scratch(G, phi, p, nodes, 64, 30, Y)
            torch.cuda.synchronize()
            out = Y.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(out))
            assert np.array_equal(out, refh)
    L = krylov.laplacian(g.n, g.rowptr, g.col, g.val)
    ora = krylov.apply("cheb", L, nodes, 30, phi, **kw).Y
    assert _rel(out, ora) < TOL32


def test_fixed_scratch_ragged_width_and_node_change(kb):
    import torch
    g = synth.random_geometric_graph(15000, 9, seed=23)
    with kb.Graph.from_csr(g) as G:
        for M, seed in [(13, 1), (7, 2)]:
            nodes = synth.sample_nodes(g.n, M, seed=seed)
            ref = torch.empty((g.n, M), dtype=torch.float32, device="cuda")
            kb.kb_krylov_apply(G, "cheb", "exp", kb.make_params(t=0.7), nodes, M, 12, ref)
            Y = torch.empty((g.n, M), dtype=torch.float32, device="cuda")
            kb.kb_cheb_apply_fixed_scratch(G, "exp", kb.make_params(t=0.7), nodes, M, 12, Y)
            torch.cuda.synchronize()
            out = Y.cpu().numpy().astype(np.float64)
            assert np.array_equal(out, ref.cpu().numpy().astype(np.float64))
            L = krylov.laplacian(g.n, g.rowptr, g.col, g.val)
            assert _rel(out, krylov.apply("cheb", L, nodes, 12, "exp", t=0.7).Y) < TOL32


def test_fixed_scratch_rejects_problems_beyond_its_size(kb):
    import torch
    g = synth.random_geometric_graph(200000, 10, seed=24)   # 3 * 200000 * 64 * 4 B > 32 MiB
    nodes = synth.sample_nodes(g.n, 64, seed=25)
    with kb.Graph.from_csr(g) as G:
        Y = torch.empty((g.n, 64), dtype=torch.float32, device="cuda")
        with pytest.raises(kb.KbError) as ei:
            kb.kb_cheb_apply_fixed_scratch(G, "exp", kb.make_params(t=1.0), nodes, 64, 10, Y)
        assert ei.value.code == -1
        assert "fixed scratch holds" in str(ei.value)


@pytest.mark.parametrize("kw", [dict(eps=float("inf"), s=1.0), dict(eps=0.1, s=float("inf")),
                                dict(eps=0.0, s=1.0), dict(eps=0.1, s=-1.0)])
def test_fixed_scratch_rejects_the_spline_parameters_kb_krylov_apply_rejects(kb, kw):
    import torch
    g = synth.random_geometric_graph(2000, 9, seed=26)
    nodes = synth.sample_nodes(g.n, 4, seed=27)
    with kb.Graph.from_csr(g) as G:
        Y = torch.empty((g.n, 4), dtype=torch.float32, device="cuda")
        for call in (kb.kb_cheb_apply_fixed_scratch, kb.kb_krylov_apply):
            with pytest.raises(kb.KbError) as ei:
                if call is kb.kb_krylov_apply:
                    call(G, "cheb", "spline", kb.make_params(**kw), nodes, 4, 8, Y)
                else:
                    call(G, "spline", kb.make_params(**kw), nodes, 4, 8, Y)
            assert ei.value.code == -1
