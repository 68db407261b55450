"""The multi-rank bench path on CPU: two gloo ranks (127.0.0.1) agree on the
slowest rank's time and on the whole-job rate of N replicas."""
from __future__ import annotations

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 100.0 + 50.0 * rank  # rank 1 is the slow one
        worst = bench.max_over_ranks(mine, dist)
        rate = bench.whole_job_rate(1000, 4, world, worst)
        dist.barrier()
        q.put((rank, worst, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, worst, rate in got:
        assert worst == 150.0
        assert rate == pytest.approx(1000 * 4 * 2 / 0.150)


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_rate(10, 2, 1, 1000.0) == pytest.approx(20.0)
