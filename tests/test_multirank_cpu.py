"""The N > 1 path of bench.py (the batch split across ranks, max-over-ranks timing, per-instance
bounds gathered at rank 0) on CPU with the gloo backend and two ranks, and the bench's
bookkeeping."""
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
    # (4 n + 12 O; the bound one also stores P, + 4 n, and reads the root values, + 4 nb)
    assert bench.algorithmic_bytes("iteration", N, O, n, nb) == 32 * N + 72 * O + 12 * n + 16 * nb
    # lane tiles: one byte of arcs per occurrence, no node offsets or successor pairs
    assert bench.algorithmic_bytes("fwd", N, O, n, nb, N, O) == 8 * N + 21 * O + 4 * nb
    assert bench.algorithmic_bytes("iteration", N, O, n, nb, N // 2, O // 3) == \
        32 * N + 72 * O + 12 * n + 16 * nb - 2 * (8 * (N // 2) + 3 * (O // 3))


def test_partition_covers_batch_once_and_balances():
    import bench
    w = [bench.batch_nnz(s) for s in range(256)]
    for world in (1, 2, 3, 8):
        parts = bench.partition_instances(w, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(256))
        loads = [sum(w[k] for k in p) for p in parts]
        # greedy heaviest-first: no rank exceeds the lightest by more than the largest instance
        assert max(loads) - min(loads) <= max(w)
        assert all(p == sorted(p) for p in parts)
    assert bench.partition_instances([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]


def _gather_worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import numpy as np

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = bench.partition_instances([3, 7, 2, 9, 4, 4, 1], world)
        mine = parts[rank]
        vals = [100.0 + k for k in mine]  # a per-instance value each rank computed
        out = bench.gather_instance_values(vals, mine, 7, world)
        total = bench.sum_over_ranks(float(len(mine)), world)
        results[rank] = (None if out is None else out.tolist(), total)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_gather_of_instance_bounds():
    world = 2
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    results = manager.dict()
    mp.start_processes(_gather_worker, args=(world, _free_port(), results), nprocs=world, start_method="spawn")
    out0, total0 = results[0]
    out1, total1 = results[1]
    assert out1 is None
    assert out0 == [100.0 + k for k in range(7)]
    assert total0 == total1 == 7.0


def test_batch_reference_assembly():
    """The CPU baseline and time-to-bound bookkeeping of the batch line on made-up traces: the
    reference bound is the oracle's where it ran, the packed time is the slowest instance's, the
    plain time sums each solver's own iterations."""
    import numpy as np

    import bench

    class FakePool:
        def __init__(self, res):
            self.res = res

        def result(self, key):
            return self.res[key]

    iters, count = 10, 4
    traj = np.tile(np.linspace(-10.0, -1.0, iters)[:, None], (1, count))
    traj[:, 2] = np.linspace(-20.0, -2.0, iters)
    finals = traj[-1].copy()
    sample = [0, 2]
    res = {("member", 0): (None, np.array([-1.0]), 2.0, 100), ("member", 2): (None, np.array([-2.0]), 4.0, 300)}
    plain = {"ms_per_solver": np.full(count, 5.0), "traces": traj.T.copy()}
    cpu, ttb = bench.batch_reference(FakePool(res), sample, iters, finals, traj, 0.5, plain)
    assert cpu["cores"] == 2 and cpu["value"] == pytest.approx(2 * 400 * iters / 4.0)
    assert cpu["per_core_value"] == pytest.approx(2 * 400 * iters / 6.0)
    assert ttb["max_rel_err_final_bound_vs_oracle"] == 0.0
    k0 = bench.first_within(traj[:, 0], -1.0 - 1e-3)
    assert ttb["sampled_instances"]["0"]["iterations"] == k0 == iters
    allv = ttb["all_instances"]
    assert allv["packed_ms"] == pytest.approx(iters * 0.5)
    assert allv["iterations_identical_plain_and_packed"]
    assert allv["plain_ms"] == pytest.approx(count * iters * 0.5)

