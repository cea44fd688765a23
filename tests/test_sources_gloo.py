"""Source-parallel misfit gradients: sources are dealt to the ranks in blocks and
the per-rank misfits and gradients are summed by one all-reduce (the only exchange
of the source-sharded path).  Host logic, run as two gloo ranks on the CPU with
per-source contributions standing in for the GPU adjoint solves."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("nsrc,world", [(16, 2), (17, 2), (3, 4), (32, 8), (1, 1), (0, 3)])
def test_every_source_belongs_to_exactly_one_rank(nsrc, world):
    from paper_2209_10886_gb300.helm import source_shard
    owned = [s for r in range(world) for s in source_shard(nsrc, r, world)]
    assert owned == list(range(nsrc))
    sizes = [len(source_shard(nsrc, r, world)) for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _contribution(s, N):
    # the misfit and gradient of source s alone (a stand-in with distinct values)
    g = torch.arange(N, dtype=torch.float64) * (s + 1) + 0.5 * s
    return 0.25 * (s + 1) ** 2, g


def _rank(rank, world, port, nsrc, N, out):
    sys.path.insert(0, ROOT)
    from paper_2209_10886_gb300.helm import reduce_misfit, source_shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        J, g = 0.0, torch.zeros(N, dtype=torch.float64)
        for s in source_shard(nsrc, rank, world):
            Js, gs = _contribution(s, N)
            J, g = J + Js, g + gs
        out[rank] = reduce_misfit(J, g)
    finally:
        dist.destroy_process_group()


def test_two_ranks_sum_misfit_and_gradient_over_all_sources():
    world, nsrc, N = 2, 7, 33
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, nsrc, N, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    Jt, gt = 0.0, torch.zeros(N, dtype=torch.float64)
    for s in range(nsrc):
        Js, gs = _contribution(s, N)
        Jt, gt = Jt + Js, gt + gs
    for rank in range(world):
        J, g = res[rank]
        assert abs(J - Jt) <= 1e-12 * abs(Jt)
        assert torch.allclose(g, gt, rtol=1e-14, atol=0)


def test_single_process_reduce_is_the_identity():
    from paper_2209_10886_gb300.helm import reduce_misfit
    g = torch.ones(4, dtype=torch.float64)
    assert reduce_misfit(2.0, g) == (2.0, g)
