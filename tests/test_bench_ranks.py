"""The multi-GPU bench path is replicas (rays are independent, the BVH is
read-only): each rank times its own copy of the workload between barriers
and the job's time is the slowest rank's.  This runs that host logic with
two gloo ranks on the CPU."""
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


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        local_ms = [120.0, 150.0][rank]  # rank 1 is the slow one
        mx = bench.max_over_ranks(local_ms, dist, "cpu")
        dist.barrier()
        value = bench.whole_job_mrays(3_000_000, 5, world, mx)
        out[rank] = (mx, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 150.0
    expect = 3_000_000 * 5 * world / 0.150 / 1e6
    assert out[0][1] == pytest.approx(expect) and out[1][1] == pytest.approx(expect)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_mrays(1_000_000, 10, 1, 1000.0) == pytest.approx(10.0)
