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
