"""Multi-rank host logic of the benchmark on CPU: two gloo ranks (replicas)
report the slowest rank's time and the sum of the ranks' units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms, units = bench.aggregate(total_ms=10.0 * (rank + 1), units=100 * (rank + 1), world=world)
        out[rank] = (ms, units)
    finally:
        dist.destroy_process_group()


def test_two_replicas_aggregate():
    ctx = mp.get_context("spawn")
    world = 2
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        ms, units = res[r]
        assert ms == 20.0                 # the slowest rank's elapsed time
        assert units == 300.0             # every rank's units
    assert 300.0 / (20.0 / 1e3) == 15000.0


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate(5.0, 7, 1) == (5.0, 7.0)
