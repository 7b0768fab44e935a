"""The replica path of bench.py (one process per GPU, no exchange on the data path) on the
CPU: two gloo ranks agree on the slowest replica's time, and the whole-job rate counts the
units of every replica over that time."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = 10.0 * (rank + 1)                      # rank 0: 10 ms, rank 1: 20 ms
    total = bench.max_over_ranks(mine, world)
    rate = bench.whole_job_rate(18, 5, world, total)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, total, rate))


def test_two_gloo_replicas_take_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, rate in got:
        assert total == 20.0                          # the slower replica's time
        assert rate == pytest.approx(2 * 18 * 5 / 0.020)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.whole_job_rate(18, 10, 1, 100.0) == pytest.approx(1800.0)
