"""The multi-GPU path is replicas only (the force phase needs no exchange on
one GPU each): bench.py's cross-rank aggregation, run as two gloo ranks on
the CPU, takes the slowest rank's step time and counts every rank's bodies."""
import os
import socket

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
    try:
        import bench

        ms, value = bench.aggregate_over_ranks(1.0 + rank, 1000, world, dist, "cpu")
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_aggregation_takes_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    slowest = 1.0 + (world - 1)
    for r in range(world):
        ms, value = out[r]
        assert ms == slowest
        assert value == pytest.approx(1000 * world / (slowest / 1e3))


def test_single_rank_needs_no_process_group():
    import bench

    ms, value = bench.aggregate_over_ranks(2.5, 4000, 1)
    assert ms == 2.5 and value == pytest.approx(4000 / 2.5e-3)
