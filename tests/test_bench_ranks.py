"""Host logic of bench.py's multi-rank path (independent replicas, one per GPU), run as two gloo
ranks on the CPU: the timed region is the slowest rank's, and the value counts every rank's
particles over that time."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    slowest = bench.max_over_ranks(times[rank], dist, "cpu")
    out.put((rank, slowest, bench.replica_rate(1000, 4, world, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_every_rank_counts():
    world = 2
    times = [12.5, 20.0]  # ms per timed region on each rank
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, slowest, rate in got:
        assert slowest == 20.0
        assert rate == pytest.approx(1000 * 4 * 2 / 0.020)


def test_single_rank_is_its_own_time():
    import bench

    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.replica_rate(1 << 24, 20, 1, 10.0) == pytest.approx((1 << 24) * 20 / 0.010)
