"""Host logic of the multi-GPU bench (replicas, one process per GPU), run as two
gloo ranks on the CPU: each rank takes its own inputs, the timing is the
slowest rank's, and the throughput counts every rank's volumes."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = 1.0 + 0.5 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(elapsed, dist, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(1000, rank))
        out[rank] = (slowest, bench.aggregate_rate(10, world, slowest), tuple(seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    world = 2
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert set(out.keys()) == {0, 1}
    for r in range(world):
        slowest, rate, seeds = out[r]
        assert slowest == 1.5
        assert rate == pytest.approx(2 * 10 / 1.5)
        assert len(set(seeds)) == world  # every replica reconstructs different phantoms


def test_single_process_helpers():
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.aggregate_rate(10, 1, 2.0) == 5.0
    assert bench.replica_seed(7, 0) == 7 and bench.replica_seed(7, 3) == 3007
