"""The serving front end (kb_server_*) and the scratch-size query, through the C ABI.

Requests run concurrently on the server's streams; each result must equal, bit for bit,
the result of the same kb_krylov_apply call made directly (same kernels, same inputs).
"""
import numpy as np
import pytest

import synth

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
def graphs(kb):
    gs = [synth.random_geometric_graph(20000, 10, seed=31),
          synth.barabasi_albert_graph(15000, 5, seed=32, weighted=True)]
    Gs = [kb.Graph.from_csr(g) for g in gs]
    yield list(zip(gs, Gs))
    for G in Gs:
        G.destroy()


def _requests():
    rng = np.random.default_rng(40)
    out = []
    methods = ["cbl", "gbl", "sbl", "cheb", "cheb2"]
    for i in range(14):
        gi = i % 2
        M = int(rng.integers(1, 129))
        method = methods[i % 5]
        if i % 3 == 0:
            phi, kw = "spline", dict(eps=float(10 ** rng.uniform(-2, -1)), s=float(rng.integers(1, 3)))
        else:
            phi, kw = "exp", dict(t=float(rng.uniform(0.1, 5.0)))
        out.append((gi, method, phi, kw, M, int(rng.integers(5, 25)), int(rng.integers(0, 1 << 30))))
    return out


def test_server_results_equal_direct_calls(kb, graphs):
    import torch
    reqs = _requests()
    outs, direct = [], []
    with kb.Server(streams=4, queue_capacity=64) as sv:
        tickets = []
        for gi, method, phi, kw, M, m, seed in reqs:
            g, G = graphs[gi]
            nodes = synth.sample_nodes(g.n, M, seed=seed)
            Y = torch.full((g.n, M), float("nan"), dtype=torch.float32, device="cuda")
            tickets.append(sv.submit(G, method, phi, kb.make_params(**kw), nodes, m, Y))
            outs.append((Y, nodes))
        lat = []
        for t in tickets:
            r = sv.poll(t, wait_ms=-1)
            assert r is not None
            info, ms = r
            assert info["status"] == 0
            lat.append(ms)
    assert all(v > 0 for v in lat)
    for (gi, method, phi, kw, M, m, seed), (Y, nodes) in zip(reqs, outs):
        g, G = graphs[gi]
        Yd = kb.kernel_columns(G, method, phi, nodes, m, **kw)
        torch.cuda.synchronize()
        assert torch.equal(Y, Yd), (method, phi, M, m)


def test_server_queue_capacity_and_budget(kb, graphs):
    import torch
    g, G = graphs[0]
    nodes = synth.sample_nodes(g.n, 8, seed=1)
    Ys = [torch.empty((g.n, 8), dtype=torch.float32, device="cuda") for _ in range(3)]
    p = kb.make_params(t=1.0)
    with kb.Server(streams=1, queue_capacity=2) as sv:
        t0 = sv.submit(G, "cbl", "exp", p, nodes, 10, Ys[0])
        t1 = sv.submit(G, "cbl", "exp", p, nodes, 10, Ys[1])
        with pytest.raises(kb.KbError) as ei:
            sv.submit(G, "cbl", "exp", p, nodes, 10, Ys[2])
        assert ei.value.code == -8
        assert sv.poll(t0, wait_ms=-1) is not None
        t2 = sv.submit(G, "cbl", "exp", p, nodes, 10, Ys[2])
        for t in (t1, t2):
            assert sv.poll(t, wait_ms=-1) is not None
        with pytest.raises(kb.KbError) as ei:
            sv.poll(t0)
        assert ei.value.code == -1   # a finished request is reported once
    need = kb.kb_workspace_bytes(G, "cbl", "exp", p, 8, 10)
    assert need > 10 * g.n * 16 * 4   # at least the 10 stored blocks of width 16
    with kb.Server(streams=2, queue_capacity=8, memory_budget=need - 1) as sv:
        with pytest.raises(kb.KbError) as ei:
            sv.submit(G, "cbl", "exp", p, nodes, 10, Ys[0])
        assert ei.value.code == -5
    # a budget for one request at a time still runs several requests (one after another)
    with kb.Server(streams=3, queue_capacity=8, memory_budget=need) as sv:
        ts = [sv.submit(G, "cbl", "exp", p, nodes, 10, Y) for Y in Ys]
        for t in ts:
            assert sv.poll(t, wait_ms=-1) is not None
    torch.cuda.synchronize()
    assert torch.equal(Ys[0], Ys[1]) and torch.equal(Ys[1], Ys[2])


def test_server_reports_solve_errors_on_poll(kb, graphs):
    import torch
    g, G = graphs[0]
    Y = torch.empty((g.n, 4), dtype=torch.float32, device="cuda")
    with kb.Server(streams=2, queue_capacity=8) as sv:
        t = sv.submit(G, "gbl", "exp", kb.make_params(t=1.0), np.array([5, 6, 6, 7]), 8, Y)
        with pytest.raises(kb.KbError) as ei:
            sv.poll(t, wait_ms=-1)
        assert ei.value.code == -3
        with pytest.raises(kb.KbError):
            sv.poll(123456)


def test_workspace_bytes_matches_layout(kb, graphs):
    g, G = graphs[0]
    p32, p64 = kb.make_params(t=1.0), kb.make_params(t=1.0, basis="f64")
    b32 = kb.kb_workspace_bytes(G, "cheb", "exp", p32, 64, 30)
    b64 = kb.kb_workspace_bytes(G, "cheb", "exp", p64, 64, 30)
    # three Clenshaw blocks of n x 64 dominate: FP64 about twice FP32
    assert 3 * g.n * 64 * 4 <= b32 < 3 * g.n * 64 * 4 * 1.2
    assert 1.9 < b64 / b32 < 2.1
    # the Lanczos methods store the basis: grows linearly in m
    c10 = kb.kb_workspace_bytes(G, "gbl", "exp", p32, 64, 10)
    c20 = kb.kb_workspace_bytes(G, "gbl", "exp", p32, 64, 20)
    assert abs((c20 - c10) - 10 * g.n * 64 * 4) < 0.05 * (c20 - c10)
    # non-integer s adds the per-node scratch of the quadrature (one block factorisation per
    # node, at most 2 x SMs nodes at a time); s >= 65 is not supported
    w_int = kb.kb_workspace_bytes(G, "cbl", "spline", kb.make_params(eps=0.1, s=2.0), 4, 5)
    w_frac = kb.kb_workspace_bytes(G, "cbl", "spline", kb.make_params(eps=0.1, s=1.5), 4, 5)
    assert w_frac > w_int
    with pytest.raises(kb.KbError):
        kb.kb_workspace_bytes(G, "cbl", "spline", kb.make_params(eps=0.1, s=65.5), 4, 5)


def test_server_falls_back_to_sbl_on_block_breakdown(kb):
    # path 0-1-2 with W = {0, 2}: the classical block process meets a rank-one block; with
    # fallback_sbl the server reruns the request as one Lanczos process per column and the
    # result equals the direct sbl call bit for bit
    import torch
    g = synth.path_graph(3)
    with kb.Graph.from_csr(g) as G:
        Y = torch.empty((3, 2), dtype=torch.float32, device="cuda")
        p = kb.make_params(t=1.0)
        with kb.Server(streams=1, queue_capacity=4) as sv:
            t = sv.submit(G, "cbl", "exp", p, np.array([0, 2]), 3, Y)
            with pytest.raises(kb.KbError) as ei:
                sv.poll(t, wait_ms=-1)
            assert ei.value.code == -6
        with kb.Server(streams=1, queue_capacity=4, fallback_sbl=True) as sv:
            t = sv.submit(G, "cbl", "exp", p, np.array([0, 2]), 3, Y)
            info, _ = sv.poll(t, wait_ms=-1)
        assert info["status"] == 0 and info["breakdown_step"] >= 0
        Yd = kb.kernel_columns(G, "sbl", "exp", [0, 2], 3, t=1.0)
        torch.cuda.synchronize()
        assert torch.equal(Y, Yd)
