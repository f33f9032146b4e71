"""The N > 1 path of bench.py (independent replicas, max-over-ranks timing) on CPU with the
gloo backend and two ranks."""
from __future__ import annotations

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, rank, world)
        ms = 10.0 + 5.0 * rank  # rank 1 is the slowest
        slow = bench.max_over_ranks(ms, world)
        results[rank] = (slow, bench.replica_throughput(1000.0, slow, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_timing():
    world = 2
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    results = manager.dict()
    mp.start_processes(_worker, args=(world, _free_port(), results), nprocs=world, start_method="spawn")
    assert results[0] == results[1]
    slow, thr = results[0]
    assert slow == pytest.approx(15.0)
    assert thr == pytest.approx(2 * 1000.0 / 0.015)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_throughput(10.0, 2.0, 1) == pytest.approx(5000.0)


def test_bench_bookkeeping():
    """Kernels per step of the per-phase schedule (four per iteration plus the kernel that
    finishes the last bound of each captured chain of 8 or 1 iterations), the staging decode of
    bdd_sizes' out[12] (two bits per sweep direction) and the algorithmic bytes of an iteration."""
    import bench
    assert bench.graph_launches(500) == 4 * 500 + 62 + 4
    assert bench.graph_launches(8) == 33 and bench.graph_launches(1) == 5
    for f in range(3):
        for b in range(3):
            class S:
                staging = f | (b << 2)
            st = bench.staging_of(S)
            assert st == {"forward": bench.STAGING[f], "backward": bench.STAGING[b]}
    N, O, n, nb = 1000, 700, 300, 90
    # the sum of the per-kernel figures: two sweeps (16 N + 24 O + 4 / 8 nb), two pending passes
    # (8 n + 12 O, the bound one + 4 nb)
    assert bench.algorithmic_bytes("iteration", N, O, n, nb) == 32 * N + 72 * O + 16 * n + 16 * nb
