"""bench.py's multi-rank timing on the CPU: two gloo ranks with different step
times agree on the slowest one, and the job rate counts every rank's steps
over that time (independent replicas, weak scaling)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    m = bench.max_over_ranks(local_ms, world, "cpu")
    out[rank] = (m, bench.job_rate(40, world, m))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        m, rate = res[r]
        assert m == 150.0
        assert rate == pytest.approx(2 * 40 / 0.150)


def test_single_rank_is_its_own_time():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(10, 1, 100.0) == pytest.approx(100.0)
