"""Multi-GPU path of the benchmark (replicas only), exercised on CPU with gloo ranks.

Every rank runs an independent replica; the only collective is the max over ranks of the
step time (host logic, no data path).  World size 2, processes started with spawn.
"""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 + 5.0 * rank            # rank 1 is the slow one
        ms = bench.job_time_ms(ms_local, world, "cpu")
        value = bench.job_value(640, world, ms)
        q.put((rank, ms, value, bench.replica_node_seed(2, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value, seed in res:
        assert ms == 15.0                        # max over ranks on every rank
        assert value == pytest.approx(2 * 640 / 0.015)
    assert res[0][3] != res[1][3]               # independent node sets per replica


def test_single_rank_needs_no_process_group():
    assert bench.job_time_ms(7.5, 1, "cpu") == 7.5
    assert bench.job_value(640, 1, 100.0) == pytest.approx(6400.0)


def test_reference_arm_only_runs_on_rank_zero(capsys):
    class A:
        pass
    bench.run_reference(A(), 1, 2)                # rank 1: returns without work or output
    assert capsys.readouterr().out == ""


def test_stream_assignment_balances_the_solves():
    import bench
    solves = [(m, t) for m in ["cbl", "gbl", "sbl", "cheb", "cheb2"] for t in (0.5, 2.0)]
    where, order = bench.assign_streams(solves, 5, "lpt")
    assert sorted(order) == list(range(len(solves)))
    load = [0.0] * 5
    for i, j in enumerate(where):
        load[j] += bench.SOLVE_COST[solves[i][0]]
    # the two long solves get a stream each; no stream carries more than the longest solve
    assert where[0] != where[1]
    assert max(load) <= bench.SOLVE_COST["cbl"] + 1e-9
    # round robin keeps the given order
    rr, rorder = bench.assign_streams(solves, 5, "rr")
    assert rr == [i % 5 for i in range(10)] and rorder == list(range(10))
    # one stream: everything in order on stream 0
    one, _ = bench.assign_streams(solves, 1, "lpt")
    assert one == [0] * 10


def test_critical_path_streams_hold_the_costliest_solves():
    import bench
    solves = [(m, t) for m in ["cbl", "gbl", "sbl", "cheb", "cheb2"] for t in (0.5, 2.0)]
    where, _ = bench.assign_streams(solves, 5, "lpt")
    hot = bench.critical_streams(solves, where)
    assert hot == {where[i] for i, (m, _) in enumerate(solves) if m == "cbl"}
    assert len(hot) == 2
    # no cbl in the step: the next costliest method marks the critical path
    s2 = [("cheb", 0.5), ("gbl", 2.0), ("cheb2", 1.0)]
    w2, _ = bench.assign_streams(s2, 3, "lpt")
    assert bench.critical_streams(s2, w2) == {w2[1]}
