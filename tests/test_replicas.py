"""The multi-GPU form of the benchmark is N independent replicas (no data-path collective): each
rank times its own steps between barriers, and rank 0 reports the units all ranks processed over the
slowest rank's time.  These tests run that host logic as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        bench.barrier(world)
        # rank r processed 1000 (r + 1) rays in 10 + r ms
        value, ms = bench.whole_job_rate(1000.0 * (rank + 1), 10.0 + rank, world)
        out[rank] = (value, ms, bench.max_over_ranks(float(rank), world), bench.sum_over_ranks(1.0, world))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_aggregation_over_gloo(world):
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    units = 1000.0 * sum(range(1, world + 1))
    slowest = 10.0 + (world - 1)
    for r in range(world):
        value, ms, mx, sm = res[r]
        assert ms == slowest
        assert value == pytest.approx(units / (slowest / 1e3), rel=1e-12)
        assert mx == world - 1 and sm == world


def test_single_rank_needs_no_process_group():
    import bench

    value, ms = bench.whole_job_rate(5000.0, 2.0, 1)
    assert ms == 2.0 and value == pytest.approx(2.5e6)
