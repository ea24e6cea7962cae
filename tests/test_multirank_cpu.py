"""bench.py --gpus N runs one replica of the step per rank (every 8x8 block
is independent; no data-path collective) and reports the whole job: the
slowest rank's time and the bytes of all ranks.  This test runs that host
logic on two gloo ranks on the CPU: both ranks get the maximum of their
times, the throughput counts both replicas, and each rank draws its own
pair of fields."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        out[rank] = (ms, bench.job_throughput(world, 1024, 4, ms), bench.replica_seeds(1024, rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_all_bytes():
    import bench

    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    per_rank = bench.step_bytes(1024) * 4 / (15.0e-3) / 1e9
    assert res[0][1] == pytest.approx(2 * per_rank)
    assert res[0][2] != res[1][2] and len({*res[0][2], *res[1][2]}) == 4
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
