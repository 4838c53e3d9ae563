"""The benchmark's multi-rank figures, on CPU with two gloo ranks: the job's
samples are the sum over ranks, its time the slowest rank's, and every rank
gets the same figures (rank 0 prints them)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    samples, elapsed = bench.aggregate_ranks(100 * (rank + 1), 1.0 + 0.5 * rank, dist, "cpu")
    out[rank] = (samples, elapsed)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_job_figures_sum_samples_and_take_the_slowest_rank(world):
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    want = (100.0 * world * (world + 1) / 2, 1.0 + 0.5 * (world - 1))
    assert all(got[r] == want for r in range(world))


def test_single_rank_figures_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(123, 4.5) == (123, 4.5)
