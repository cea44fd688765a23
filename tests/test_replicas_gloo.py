"""The multi-GPU path of bench.py is replicas only (independent sources, no
collective on the data path): its host-side bookkeeping, the max-over-ranks
time and the whole-job throughput, run here as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [120.0, 150.0][rank]                      # the second replica is slower
        slowest = bench.max_over_ranks(ms, world, torch.device("cpu"))
        out[rank] = (slowest, bench.job_throughput(1000, world, slowest))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time_and_the_whole_job_throughput():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        slowest, value = res[rank]
        assert slowest == 150.0
        assert value == pytest.approx(2 * 1000 / 0.150)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, 1, None) == 7.0
    assert bench.job_throughput(10, 1, 1000.0) == pytest.approx(10.0)
