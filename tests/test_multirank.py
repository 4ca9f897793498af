"""The benchmark's multi-process aggregation on CPU (gloo, world size 2): every rank's units are
summed and divided by the slowest rank's time, as the contract for N GPUs asks. The path itself
shards as independent replicas, so this host logic is the whole of the multi-GPU code."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r processed 100 (r + 1) units in 0.010 (r + 1) s
        rate, slowest = bench.job_rate(100.0 * (rank + 1), 0.010 * (rank + 1))
        out[rank] = (rate, slowest)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_rate_sums_units_over_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        rate, slowest = out[rank]
        assert slowest == pytest.approx(0.020)
        assert rate == pytest.approx((100.0 + 200.0) / 0.020)


def test_job_rate_single_process_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    rate, s = bench.job_rate(5406 * 200, 0.04)
    assert s == 0.04 and rate == pytest.approx(5406 * 200 / 0.04)
