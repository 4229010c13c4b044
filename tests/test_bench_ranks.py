"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
step time; every rank must see the slowest time, and the whole-job value is
world x units / slowest time (replicas, weak scaling)."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [2.5, 4.0][rank]
        slowest = bench.max_over_ranks(mine, dist, "cpu")
        q.put((rank, slowest, bench.whole_job_value(1000, world, slowest)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value in got:
        assert slowest == 4.0
        assert value == pytest.approx(2 * 1000 / 4.0e-3)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.whole_job_value(500, 1, 2.0) == pytest.approx(250000.0)
