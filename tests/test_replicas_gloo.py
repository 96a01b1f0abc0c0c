"""The multi-GPU path is replicas only (every rank fits its own data set, no exchange step):
its host logic - the whole-job aggregate over ranks (slowest rank's time, FLOPs summed) and the
per-rank data sets - checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    import synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r: 100 + 50 r ms, (r + 1) * 1e12 FLOPs, (r + 1) * 2e12 nominal
        t, f, n = bench.aggregate_over_ranks(100.0 + 50.0 * rank, (rank + 1) * 1e12, (rank + 1) * 2e12, world,
                                             torch.device("cpu"))
        w = synth.small_mixture(rank)  # replicas fit their own data (seed + rank)
        out[rank] = (t, f, n, float(w.X[0, :4].sum()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, f, n, _ = out[r]
        assert t == 150.0  # slowest rank
        assert f == 3e12 and n == 6e12  # summed over the replicas
    assert out[0][3] != out[1][3]  # different data set per rank


def test_single_rank_is_identity():
    import bench

    assert bench.aggregate_over_ranks(12.5, 7.0, 9.0, 1, None) == (12.5, 7.0, 9.0)
