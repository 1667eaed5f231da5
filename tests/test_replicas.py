"""The multi-GPU path is replicas only: each rank solves its own instance, and the bench
reports the slowest rank's step time and all ranks' updates over it. Checked with two gloo
ranks on the CPU (the aggregation is the only cross-rank step)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.replica_throughput(10.0 + 5.0 * rank, 1.0e9, world, "cpu")
    dist.barrier()
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_gloo_replicas_report_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == pytest.approx(15.0)
        assert value == pytest.approx(1.0e9 * world / 0.015)


def test_single_rank_is_unchanged():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    assert bench.replica_throughput(20.0, 1e9, 1, "cpu") == (20.0, pytest.approx(5e10))
