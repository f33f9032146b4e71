#!/usr/bin/env python
"""Benchmark of the dual iteration (forward sweep, pending sums, backward sweep, pending sums with
the FP64 bound) on the batch of 256 uneven Potts MRF instances (grids 16x16 .. 128x128, 2 .. 8
labels, packed block-diagonally into one solver; 200 iterations per step).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config C]

A step is one full run of the workload's 200 iterations from the initial multipliers (the solver
restarts before each step, outside the timed region).  Every iteration moves about 38 GB, far more
than L2, so no flush is needed between steps.  value = BDD arcs processed per second (2 x nodes x
iterations per step, all ranks) from CUDA events on the launching stream.  Under torchrun each
rank packs its share of the 256 instances (balanced by coefficient count) and the ranks never
exchange data on the path.

Beside the headline the line carries: the roofline of the dominant kernel; the oracle on the host
cores on a sample of the batch (CPU baseline and the reference bounds of the time-to-bound);
the packed solve's per-instance time to a bound within 1e-3 of the oracle's; the plain form (one
solver per instance, iterated one after another) at the same accuracy; end to end through the C
ABI with host buffers; and, per form the benchmark spec names (plain on the MRF, matching,
tomography and tracking workloads; smoothed with the adjoint on tracking), arcs/s and the time to
1e-3 of the oracle's bound.  `--config C` (0..3) prints a line for one single-instance workload
instead; `--impl reference` times the FP64 oracle on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

from instances import CONFIG_ITERS, CONFIG_NAMES, config  # noqa: E402

METRIC = "dual-iter BDD arcs/s & time to oracle bound+-1e-3, plain vs batched/diff"
UNIT = "arcs/s"
TTB_TOL = 1e-3
BATCH_COUNT = 256
SAMPLE_EVERY = 32        # the oracle runs every 32nd instance of the batch (8 instances)
SMOOTH_TAU = 0.1


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--iters", type=int, default=0, help="iterations per step (default: the workload's)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle runs on the host cores")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-solver-per-instance loop")
    ap.add_argument("--no-forms", action="store_true", help="skip the per-form time-to-bound table")
    ap.add_argument("--oracle-workers", type=int, default=12, help="host processes running the oracle")
    ap.add_argument("--schedule", type=int, default=1, help="1 per-phase graphs (default), 0 persistent kernel")
    ap.add_argument("--staging", type=int, default=-1,
                    help="warp-tile staging of the update sweeps: -1 autotuned (default), 0 bulk-copy ring, "
                         "1 8-layer cp.async windows, 2 the same double-buffered")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT, help="instances in the batch workload")
    ap.add_argument("--variant-iters", type=int, default=300)
    ap.add_argument("--variants-only", action="store_true", help="print only the order / averaging comparison")
    ap.add_argument("--split-only", action="store_true", help="print only the sub-BDD comparison")
    ap.add_argument("--smoothed-only", action="store_true",
                    help="print only the smoothed bound with its adjoint (tracking 50x200, K = 50)")
    ap.add_argument("--split-iters", type=int, default=200, help="timed iterations per sub-BDD variant")
    ap.add_argument("--split-ttb-iters", type=int, default=300,
                    help="oracle iterations giving the sub-BDD comparison's target bound (the GPU runs 3x)")
    return ap.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


# ------------------------------------------------------------------------------------------
# algorithmic bytes per kernel launch (minimum traffic of the slab layout: every array a kernel
# needs, touched once)
# ------------------------------------------------------------------------------------------
def graph_launches(iters: int) -> int:
    """Kernels the per-phase schedule launches for `iters` iterations: four per iteration (two
    sweeps, two pending passes), plus the one-warp kernel that finishes the last bound of each
    captured chain (chains of 8 iterations, then single iterations)."""
    return 4 * iters + iters // 8 + iters % 8


def algorithmic_bytes(kind: str, N: int, O: int, n: int, nb: int, lane_N: int = 0, lane_O: int = 0) -> int:
    """Bytes a kernel must move once per launch; lane_N / lane_O: nodes and occurrences of the
    lane tiles (bdd_sizes [18] / [17]), whose arcs are one byte per occurrence."""
    if kind in ("fwd", "bwd"):
        # warp teams and block tiles, per node: lo/hi 8 B, fm 4 B, bm 4 B; per occurrence: node
        # offset 4, lambda read+write 8, share 4, slot 4, difference write 4.  Lane tiles, per
        # node: fm 4, bm 4; per occurrence: lane code 1, lambda 8, share 4, slot 4, difference 4.
        # Per BDD: depth (+ root value on the backward sweep)
        tN, tO = N - lane_N, O - lane_O
        return 16 * tN + 24 * tO + 8 * lane_N + 21 * lane_O + (4 if kind == "fwd" else 8) * nb
    if kind == "pending":
        # per variable: slot range 4 (P is stored by the bound pass only); per slot: difference
        # 4, occurrence id 4, share write 4
        return 4 * n + 12 * O
    if kind == "pending_bound":
        # and P write 4 per variable, root value 4 per BDD
        return algorithmic_bytes("pending", N, O, n, nb) + 4 * n + 4 * nb
    if kind == "iteration":
        return sum(algorithmic_bytes(k, N, O, n, nb, lane_N, lane_O) for k in ("fwd", "pending", "bwd", "pending_bound"))
    raise ValueError(kind)


def solver_bytes(kind: str, s) -> int:
    """algorithmic_bytes of a solver's layout."""
    return algorithmic_bytes(kind, s.N, s.O, s.n, s.nb, getattr(s, "lane_N", 0), getattr(s, "lane_O", 0))


STAGING = {0: "bulk-copy ring, 4-layer windows", 1: "8-layer cp.async windows",
           2: "double-buffered 8-layer cp.async windows"}
KINDS = ["fwd", "pending", "bwd", "pending_bound"]


def staging_of(s) -> dict:
    """Warp-tile staging the solver's autotuner chose for each update sweep."""
    return {"forward": STAGING[s.staging & 3], "backward": STAGING[(s.staging >> 2) & 3]}


def sweep_kernel_name(kind: str, s) -> str:
    """The sweep kernel as the solver runs it: lane tiles (if its layout has them) and the
    staging of its other warp tiles."""
    st = staging_of(s)
    lanes = "lane tiles + " if getattr(s, "lanes", 0) else ""
    return {"fwd": f"sweep_kernel<forward, update> ({lanes}{st['forward']})",
            "bwd": f"sweep_kernel<backward, update> ({lanes}{st['backward']})",
            "pending": "pending_kernel", "pending_bound": "pending_kernel<bound>"}[kind]


def sources_sha256() -> str:
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(HERE, "paper_2009_00481_gb300", "csrc", "*"))):
        if f.endswith((".cu", ".cpp", ".h", ".cuh")):
            with open(f, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def dram_traffic(workload: str, kernel: str, nodes: int):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary, scaled by
    node count; None when no capture exists or the CUDA sources changed since it was taken."""
    path = os.path.join(HERE, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    want_hash, found = None, None
    for line in open(path):
        line = line.strip()
        if line.startswith("# sources-sha256:"):
            want_hash = line.split(":", 1)[1].strip()
        elif line and not line.startswith("#"):
            parts = [x.strip() for x in line.split("|")]
            if len(parts) == 4 and parts[0] == workload and parts[1] == kernel:
                found = int(parts[2]) * nodes / int(parts[3])
    if found is None or want_hash != sources_sha256():
        return None
    return found


def max_over_ranks(ms: float, world: int, device: str = "cpu") -> float:
    """Step time of the slowest rank (all ranks call this; needs an initialised process group
    when world > 1)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_step_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job throughput of `world` ranks that each process the same number of units: all
    ranks' units over the slowest rank's time."""
    return world * units_per_step_per_rank / (ms_max / 1e3)


def sum_over_ranks(x: float, world: int, device: str = "cpu") -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------------------------------
# the batch: instance sizes and their split across ranks
# ------------------------------------------------------------------------------------------
def batch_nnz(s: int) -> int:
    """Nonzero coefficients of batch instance s (one-hot rows side^2 x L, two marginalisation
    rows of L + 1 coefficients per edge and label): the input size, used to balance ranks."""
    from instances import potts_batch_shape
    side, L = potts_batch_shape(s)
    E = 2 * side * (side - 1)
    return side * side * L + E * 2 * L * (L + 1)


def partition_instances(weights, world: int):
    """Instances of the batch for each rank: the heaviest instance first goes to the rank with
    the least weight so far (ties: lower rank); each rank's list ascending.  Deterministic."""
    order = sorted(range(len(weights)), key=lambda k: (-weights[k], k))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += weights[k]
    return [sorted(p) for p in parts]


def gather_instance_values(values, mine, count: int, world: int):
    """Per-instance values of every rank at rank 0, in instance order (rank 0 gets the full
    array, the others None).  Host objects only: no exchange on the iteration path."""
    if world <= 1:
        out = np.full(count, np.nan)
        out[np.asarray(mine, np.int64)] = values
        return out
    import torch.distributed as dist
    got = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object((list(mine), [float(v) for v in values]), got, dst=0)
    if dist.get_rank() != 0:
        return None
    out = np.full(count, np.nan)
    for idx, vals in got:
        out[np.asarray(idx, np.int64)] = vals
    return out


def measured_peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"bdd_bench_clocks_rank{device_index}.csv")
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(device_index), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------
# CPU side: the oracle in host processes (reference bounds, CPU baseline)
# ------------------------------------------------------------------------------------------
def _task_instance(spec):
    from instances import potts_batch_member, tomography
    kind = spec[0]
    if kind == "member":
        return potts_batch_member(spec[1])
    if kind == "config":
        return config(spec[1])
    if kind == "tomography_tie_break":
        return tomography(side=64, seed=0, unary_sigma=0.01)
    raise ValueError(spec)


def oracle_task(spec, iters: int, alpha: float = 0.0):
    """One oracle run in a host process: the deferred-averaging schedule from the initial
    multipliers for `iters` iterations (smoothed with alpha > 0), single-threaded FP64, timed
    around the iteration loop.  Returns (spec, bound trace, seconds, nodes)."""
    import oracle
    from oracle import Oracle
    oracle.build()
    o = Oracle(_task_instance(spec))
    if alpha > 0:
        o.set_alpha(alpha)
    t0 = time.perf_counter()
    tr = o.run_parallel(iters, omega=0.5)
    sec = time.perf_counter() - t0
    return spec, tr, sec, o.N


class OraclePool:
    """Oracle runs in spawned host processes, started before the GPU work and collected after
    it (they share no state with the GPU path)."""

    def __init__(self, workers: int):
        import concurrent.futures as cf
        import multiprocessing as mp
        import oracle
        oracle.build()  # compile once here, not in every worker
        self.ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
        self.jobs = {}

    def submit(self, key, spec, iters, alpha=0.0):
        self.jobs[key] = self.ex.submit(oracle_task, spec, iters, alpha)

    def result(self, key):
        return self.jobs[key].result()

    def close(self):
        self.ex.shutdown(wait=True)


def first_within(trace, target):
    """1-based iteration at which a bound trace first reaches `target`, or None."""
    hit = np.nonzero(np.asarray(trace) >= target)[0]
    return int(hit[0]) + 1 if hit.size else None


def ttb_target(lb_ref: float) -> float:
    return lb_ref - TTB_TOL * abs(lb_ref)


# ------------------------------------------------------------------------------------------
# the headline: the packed batch
# ------------------------------------------------------------------------------------------
def timed_steps(torch, s, inst, iters, steps, warmup, stream, trace):
    """`warmup` untimed steps, then `steps` steps bracketed by events; the solver restarts from
    the initial multipliers before every step (untimed).  Returns ms per step."""
    for _ in range(warmup):
        s.set_costs(inst.c)
        s.iterate_device(iters, trace=trace, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        s.set_costs(inst.c)
        evs[i][0].record(stream)
        s.iterate_device(iters, trace=trace, stream=stream.cuda_stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in evs]))


def roofline_of(s, iters, kms, peak, peak_kind, workload, label=None):
    """Roofline of the dominant per-phase kernel from the kernel-by-kernel event timings."""
    dom = int(np.argmax(kms))
    abytes = solver_bytes(KINDS[dom], s)
    per_launch_ms = float(kms[dom] / iters)
    achieved = abytes / (per_launch_ms / 1e3) / 1e9
    iter_bytes = solver_bytes("iteration", s)
    iter_ms = float(kms.sum() / iters)
    name = sweep_kernel_name(KINDS[dom], s)
    out = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
           "unit": "GB/s", "frac": achieved / peak, "traffic": dram_traffic(workload, name, s.N),
           "algorithmic_bytes_per_launch": abytes, "launch_ms": per_launch_ms,
           "iteration": {"algorithmic_bytes": iter_bytes, "ms": iter_ms,
                         "achieved_gbs": iter_bytes / (iter_ms / 1e3) / 1e9,
                         "frac": iter_bytes / (iter_ms / 1e3) / 1e9 / peak},
           "per_phase_kernel_ms_per_iteration": {k: float(v / iters) for k, v in zip(KINDS, kms)}}
    if label:
        out["note"] = label
    return out


def run_batch(args):
    import torch
    import torch.distributed as dist

    from instances import potts_batch
    from paper_2009_00481_gb300 import Solver

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if world > 1:
            dist.barrier()

    count = args.batch_count
    iters = args.iters or CONFIG_ITERS[4]
    weights = [batch_nnz(s_) for s_ in range(count)]
    mine = partition_instances(weights, world)[rank]
    sample = list(range(0, count, SAMPLE_EVERY))

    # oracle runs on the host cores, concurrently with the GPU work (1-GPU runs)
    pool = None
    if world == 1 and not args.no_cpu_baseline:
        pool = OraclePool(args.oracle_workers)
        for s_ in sample:
            pool.submit(("member", s_), ("member", s_), iters)
        if not args.no_forms:
            for k in (0, 1, 3):
                pool.submit(("plain", k), ("config", k), CONFIG_ITERS[k])
            pool.submit(("plain", 2), ("tomography_tie_break",), CONFIG_ITERS[2])
            pool.submit(("smoothed", 3), ("config", 3), CONFIG_ITERS[3], SMOOTH_TAU)

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    inst = potts_batch(seeds=mine)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    s = Solver(inst, omega=0.5, stream=stream.cuda_stream, schedule=args.schedule, staging=args.staging)
    build_s = time.perf_counter() - t0
    arcs_per_step = 2 * s.N * iters
    trace = torch.zeros(iters, dtype=torch.float64, device="cuda")

    sampler = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ms_mine = timed_steps(torch, s, inst, iters, args.steps, args.warmup, stream, trace)
    barrier()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    ms = max_over_ranks(ms_mine, world, device="cuda")
    arcs_all = sum_over_ranks(arcs_per_step, world, device="cuda")
    value = arcs_all / (ms / 1e3)

    # per-instance bounds after each iteration (untimed rerun, one iteration at a time)
    s.set_costs(inst.c)
    traj = np.zeros((iters, len(mine)))
    for it in range(iters):
        s.iterate_device(1, stream=stream.cuda_stream)
        traj[it] = s.bound_parts(inst.row_parts, inst.var_parts)
    final_mine = traj[-1]

    # kernel-by-kernel timings for the roofline of the dominant kernel
    s.set_costs(inst.c)
    kms = s.iterate_profiled(iters)
    peak, peak_kind = measured_peaks()
    roof = roofline_of(s, iters, kms, peak, peak_kind, CONFIG_NAMES[4])

    # end to end through the C ABI with host buffers: bdd_build (host BDD compile + upload +
    # autotune) from the host arrays, bdd_iterate returning the bound, multipliers and
    # min-marginals to the host, bdd_free
    e2e = None
    if args.e2e_steps > 0:
        times = []
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            s2 = Solver(inst, omega=0.5, schedule=args.schedule, staging=args.staging)
            s2.iterate(iters, lam=True, mm=True)
            s2.close()
            times.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(float(np.mean(times)), world, device="cuda")
        h2d = (inst.row_ptr.nbytes + inst.col.nbytes + inst.val.nbytes + inst.b.nbytes
               + inst.sense.nbytes + inst.c.nbytes)
        d2h = 8 + 3 * 4 * inst.nnz
        e2e = {"value": arcs_all / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(sum_over_ranks(h2d, world, device="cuda")),
               "d2h_bytes_per_step": int(sum_over_ranks(d2h, world, device="cuda")),
               "s_per_step": e2e_s,
               "includes": "bdd_build from host arrays (host BDD compile, upload, autotune) + bdd_iterate of "
                           f"{iters} iterations returning the bound, multipliers and min-marginals to the host "
                           "+ bdd_free"}

    finals = gather_instance_values(final_mine, mine, count, world)
    if rank != 0:
        s.close()
        if world > 1:
            dist.destroy_process_group()
        return

    # the plain form: one solver per instance, iterated one after another (1 GPU)
    plain = None
    if world == 1 and not args.no_plain:
        plain = run_plain_loop(args, torch, stream, iters)

    cpu, ttb = None, None
    if pool is not None:
        cpu, ttb = batch_reference(pool, sample, iters, finals, traj if world == 1 else None, ms / iters, plain)

    forms = None
    if world == 1 and not args.no_forms:
        forms = run_forms(args, torch, stream, pool)
    if pool is not None:
        pool.close()

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": CONFIG_NAMES[4], "instances": count, "iterations_per_step": iters,
                   "instances_this_rank": len(mine), "bdds": s.nb, "nodes": s.N, "arcs": 2 * s.N,
                   "arcs_all_ranks": arcs_all / iters, "occurrences": s.O, "variables": s.n, "omega": 0.5,
                   "device_bytes": s.device_bytes,
                   "l2": "inputs larger than L2 (no flush): "
                         f"{solver_bytes('iteration', s) / 1e9:.1f} GB moved per iteration",
                   "generate_s": gen_s, "build_s": build_s,
                   "parallelism": f"instances split over {world} ranks, no exchange" if world > 1 else "single"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "time_to_bound": ttb,
        "plain_loop": None if plain is None else {k: v for k, v in plain.items()
                                                  if k not in ("traces", "ms_per_solver")},
        "forms": forms,
        "gpu_launches": args.steps * graph_launches(iters),
        "schedule": "persistent" if s.schedule == 0 else "per-phase graphs",
        "staging": staging_of(s),
        "clocks": clocks,
        "wall_s": wall,
    }
    s.close()
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_plain_loop(args, torch, stream, iters):
    """The plain single-instance form on the same GPU: one solver per batch instance, each
    iterated `iters` times, one after another (one warm-up pass, then one timed pass); every
    solver's own bound trace and device ms."""
    from instances import potts_batch_member
    from paper_2009_00481_gb300 import Solver

    count = args.batch_count
    t0 = time.perf_counter()
    members = [potts_batch_member(k) for k in range(count)]
    solvers = [Solver(m, omega=0.5, stream=stream.cuda_stream, schedule=args.schedule) for m in members]
    build_s = time.perf_counter() - t0
    traces = torch.zeros((count, iters), dtype=torch.float64, device="cuda")
    for k, t in enumerate(solvers):  # warm-up (captures the graphs)
        t.iterate_device(iters, trace=traces[k], stream=stream.cuda_stream)
    for m, t in zip(members, solvers):
        t.set_costs(m.c)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(count + 1)]
    ev[0].record(stream)
    for k, t in enumerate(solvers):
        t.iterate_device(iters, trace=traces[k], stream=stream.cuda_stream)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    per = np.array([ev[k].elapsed_time(ev[k + 1]) for k in range(count)])
    total = ev[0].elapsed_time(ev[count])
    nodes = sum(t.N for t in solvers)
    for t in solvers:
        t.close()
    return {"value": 2 * nodes * iters / (total / 1e3), "unit": UNIT, "ms": total, "build_s": build_s,
            "form": f"{count} solvers, one per instance, {iters} iterations each, one after another",
            "ms_per_solver": per, "traces": traces.cpu().numpy()}


def batch_reference(pool, sample, iters, finals, traj, ms_iter, plain):
    """CPU baseline and time-to-bound of the batch from the oracle runs on the sampled
    instances."""
    runs = {s_: pool.result(("member", s_)) for s_ in sample}
    wall = max(r[2] for r in runs.values())
    arcs = sum(2 * r[3] * iters for r in runs.values())
    cpu_sec = sum(r[2] for r in runs.values())
    cpu = {"value": arcs / wall, "unit": UNIT, "cores": len(sample), "kind": "oracle",
           "per_core_value": arcs / cpu_sec,
           "sample": f"instances {sample} of the batch (every {SAMPLE_EVERY}th), {iters} iterations each from "
                     f"the initial multipliers, FP64, one host process per instance run side by side "
                     f"({cpu_sec:.1f} s of CPU work); value = their arcs over the longest run's time"}
    ref = {s_: float(r[1][-1]) for s_, r in runs.items()}
    parity = {s_: abs(finals[s_] - ref[s_]) / max(1.0, abs(ref[s_])) for s_ in sample}
    ttb = {"tolerance": TTB_TOL, "reference": "the oracle's bound after the same iterations",
           "max_rel_err_final_bound_vs_oracle": max(parity.values())}
    if traj is None:
        return cpu, ttb
    per = {}
    for s_ in sample:
        k = first_within(traj[:, s_], ttb_target(ref[s_]))
        per[str(s_)] = {"oracle_bound": ref[s_], "gpu_bound": float(finals[s_]), "iterations": k,
                        "ms_packed": k * ms_iter if k else None, "oracle_s": runs[s_][2]}
    ttb["sampled_instances"] = per
    hit = [v["iterations"] for v in per.values()]
    ttb["packed_ms_until_every_sampled_instance"] = (max(hit) * ms_iter) if all(hit) else None
    # every instance: the oracle's bound where it ran, elsewhere the packed solve's own bound
    # after the step's iterations (which the sample shows to match the oracle's to the figure above)
    refs = np.array(finals, np.float64)
    for s_ in sample:
        refs[s_] = ref[s_]
    k_all = [first_within(traj[:, k], ttb_target(refs[k])) for k in range(len(refs))]
    if not all(k_all):
        ttb["all_instances"] = {"reached": int(sum(1 for k in k_all if k)), "of": len(k_all)}
        return cpu, ttb
    ttb["all_instances"] = {
        "reference": "oracle bound on the sampled instances, elsewhere the packed solve's own final bound",
        "iterations": {"median": float(np.median(k_all)), "max": int(max(k_all)), "min": int(min(k_all))},
        "packed_ms": max(k_all) * ms_iter}
    if plain is not None:
        ms_solver = plain["ms_per_solver"] / iters
        k_plain = [first_within(plain["traces"][k], ttb_target(refs[k])) for k in range(len(refs))]
        if all(k_plain):
            plain_ms = float(sum(kk * m for kk, m in zip(k_plain, ms_solver)))
            ttb["all_instances"].update({
                "plain_ms": plain_ms, "plain_over_packed": plain_ms / (max(k_all) * ms_iter),
                "iterations_identical_plain_and_packed": bool(k_plain == k_all),
                "note": "packed: all instances iterate together until the slowest reaches its target; plain: "
                        "each solver iterates until its own instance reaches its target, one after another"})
    return cpu, ttb


# ------------------------------------------------------------------------------------------
# the other forms: plain single instances and the smoothed bound with its adjoint
# ------------------------------------------------------------------------------------------
def run_forms(args, torch, stream, pool):
    """Per form: device arcs/s, the time to within 1e-3 of the oracle's bound after the
    workload's iterations, the HBM fraction of an iteration (these working sets fit in L2:
    latency-bound), and the oracle on one host core for the same iterations."""
    from instances import tomography
    from paper_2009_00481_gb300 import Solver, binding

    peak, _ = measured_peaks()
    out = {}
    for k in (0, 1, 2, 3):
        inst = tomography(side=64, seed=0, unary_sigma=0.01) if k == 2 else config(k)
        iters = CONFIG_ITERS[k]
        s = Solver(inst, omega=0.5, stream=stream.cuda_stream)
        trace = torch.zeros(iters, dtype=torch.float64, device="cuda")
        ms = timed_steps(torch, s, inst, iters, 3, 2, stream, trace)
        tr = trace.cpu().numpy()
        ib = solver_bytes("iteration", s)
        row = {"workload": CONFIG_NAMES[k] + (" (unaries N(0, 0.01))" if k == 2 else ""), "iterations": iters,
               "nodes": s.N, "ms": ms, "value": 2 * s.N * iters / (ms / 1e3), "unit": UNIT,
               "hbm_frac": ib * iters / (ms / 1e3) / 1e9 / peak,
               "hbm_note": f"L2-resident ({ib / 1e6:.1f} MB per iteration), latency-bound",
               "gpu_bound": float(tr[-1])}
        if pool is not None:
            _, otr, osec, _ = pool.result(("plain", k))
            kk = first_within(tr, ttb_target(float(otr[-1])))
            row.update({"oracle_bound": float(otr[-1]), "iterations_to_bound": kk,
                        "ms_to_bound": ms * kk / iters if kk else None,
                        "oracle_s": osec, "oracle_value": 2 * s.N * iters / osec, "oracle_cores": 1})
        out[f"plain_{CONFIG_NAMES[k]}"] = row
        s.close()

    out.update(run_smoothed(args, torch, stream, pool))
    if pool is not None:  # the oracle's OpenMP build on all host cores, after the pool is done
        for k in (0, 1, 2, 3):
            row = out[f"plain_{CONFIG_NAMES[k]}"]
            try:
                sec, cores = oracle_omp_seconds(k)
                row.update({"oracle_omp_s": sec, "oracle_omp_value": 2 * row["nodes"] * CONFIG_ITERS[k] / sec,
                            "oracle_omp_cores": cores})
            except Exception as e:  # no OpenMP runtime on this host
                row["oracle_omp"] = f"unavailable: {e}"
    return out


def oracle_omp_seconds(k: int):
    """Seconds of the oracle's OpenMP build (schedule P's loops over BDDs and variables on all
    host cores; the same results bit for bit) for workload k's iterations, and the cores used."""
    from instances import tomography
    from oracle import Oracle, load_omp
    inst = tomography(side=64, seed=0, unary_sigma=0.01) if k == 2 else config(k)
    o = Oracle(inst, lib=load_omp())
    t0 = time.perf_counter()
    o.run_parallel(CONFIG_ITERS[k], omega=0.5)
    return time.perf_counter() - t0, int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_smoothed(args, torch, stream, pool, reps: int = 3) -> dict:
    """The smoothed bound with its adjoint (tracking 50x200, tau = 0.1, K = 50): forward and
    forward + adjoint ms, and the iterations and ms to 1e-3 of the oracle's smoothed bound."""
    from paper_2009_00481_gb300 import Solver, binding

    out = {}
    inst = config(3)
    K = CONFIG_ITERS[3]
    sm = Solver(inst, omega=0.5, stream=stream.cuda_stream, alpha=SMOOTH_TAU)
    trace = torch.zeros(K, dtype=torch.float64, device="cuda")
    sm.iterate_device(K, trace=trace, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    tr = trace.cpu().numpy()
    c = torch.tensor(inst.c, device="cuda")
    bound = torch.zeros((), dtype=torch.float64, device="cuda")
    gbound = torch.ones((), dtype=torch.float64, device="cuda")
    grad = torch.zeros(inst.n, dtype=torch.float32, device="cuda")
    sp = stream.cuda_stream

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_fwd = timed(lambda: binding.bdd_smooth_forward(sm.h, K, c.data_ptr(), bound.data_ptr(), sp))

    def fwd_bwd():
        gen = binding.bdd_smooth_forward(sm.h, K, c.data_ptr(), bound.data_ptr(), sp)
        binding.bdd_smooth_backward(sm.h, gen, gbound.data_ptr(), grad.data_ptr(), sp)

    ms_fb = timed(fwd_bwd)
    row = {"workload": CONFIG_NAMES[3], "tau": SMOOTH_TAU, "iterations": K, "nodes": sm.N,
           "ms_forward": ms_fwd, "ms_forward_and_adjoint": ms_fb,
           "value": 2 * sm.N * K / (ms_fb / 1e3), "unit": UNIT,
           "value_note": "arcs of the K smoothed iterations over the time of forward plus adjoint",
           "gpu_bound": float(tr[-1])}
    if pool is not None:
        _, otr, osec, _ = pool.result(("smoothed", 3))
        kk = first_within(tr, ttb_target(float(otr[-1])))
        row.update({"oracle_bound": float(otr[-1]), "iterations_to_bound": kk,
                    "ms_to_bound": ms_fb * kk / K if kk else None,
                    "ms_to_bound_note": "forward plus adjoint cost per iteration x iterations to the bound",
                    "oracle_s": osec, "oracle_cores": 1})
    out[f"smoothed_adjoint_{CONFIG_NAMES[3]}"] = row
    sm.close()
    return out


# ------------------------------------------------------------------------------------------
# one single-instance workload as the line (--config 0..3)
# ------------------------------------------------------------------------------------------
def run_single(args):
    import torch

    from paper_2009_00481_gb300 import Solver

    torch.cuda.set_device(0)
    k = args.config
    iters = args.iters or CONFIG_ITERS[k]
    inst = config(k)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = Solver(inst, omega=0.5, stream=stream.cuda_stream, schedule=args.schedule, staging=args.staging)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    trace = torch.zeros(iters, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        s.set_costs(inst.c)
        s.iterate_device(iters, trace=trace, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        s.set_costs(inst.c)
        flush.zero_()
        evs[i][0].record(stream)
        s.iterate_device(iters, trace=trace, stream=stream.cuda_stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    tr = trace.cpu().numpy()
    s.set_costs(inst.c)
    kms = s.iterate_profiled(iters)
    peak, peak_kind = measured_peaks()
    import oracle
    from oracle import Oracle
    oracle.build()
    o = Oracle(inst)
    t0 = time.perf_counter()
    otr = o.run_parallel(iters, omega=0.5)
    osec = time.perf_counter() - t0
    kk = first_within(tr, ttb_target(float(otr[-1])))
    out = {"metric": METRIC, "value": 2 * s.N * iters / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": CONFIG_NAMES[k], "iterations_per_step": iters, "bdds": s.nb, "nodes": s.N,
                      "l2": "flushed before each step (256 MiB write)", "parallelism": "single"},
           "roofline": roofline_of(s, iters, kms, peak, peak_kind, CONFIG_NAMES[k],
                                   "L2-resident working set: latency-bound, the HBM fraction is small by construction"),
           "time_to_bound": {"oracle_bound": float(otr[-1]), "gpu_bound": float(tr[-1]), "iterations": kk,
                             "ms": ms * kk / iters if kk else None},
           "cpu_baseline": {"value": 2 * s.N * iters / osec, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"full {CONFIG_NAMES[k]} instance, {iters} iterations, FP64 single thread"},
           "gpu_launches": args.steps * graph_launches(iters), "staging": staging_of(s), "clocks": clocks}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------------------
# variable order / averaging, and sub-BDDs (separate lines)
# ------------------------------------------------------------------------------------------
def run_variants(args, stream) -> dict:
    """Variable order (index vs Cuthill-McKee, Appendix A.3) x averaging (eq. mma-update vs SRMP,
    Appendix A.4) on the MRF workload (Potts 20x20 grid, 3 labels) and the cell-tracking-shaped
    flow ILP (50 frames x 200 detections), where the paper reorders variables: bound after
    --variant-iters iterations, iterations until the bound is within 1e-3 (relative) of the best
    final bound of the four variants, and device ms per iteration."""
    import torch

    from paper_2009_00481_gb300 import Solver, cuthill_mckee

    K = args.variant_iters
    out = {"iterations": K, "target_tol": TTB_TOL}
    for k in (0, 3):
        inst = config(k)
        cm = cuthill_mckee(inst)
        trace = torch.zeros(K, dtype=torch.float64, device="cuda")
        res = {}
        for order, rank in (("index", None), ("cm", cm)):
            for avg, name in ((0, "mma"), (1, "srmp")):
                s = Solver(inst, omega=0.5, stream=stream.cuda_stream, rank=rank, averaging=avg)
                s.iterate_device(K, trace=trace, stream=stream.cuda_stream)  # warm-up (graphs)
                s.set_costs(inst.c)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                s.iterate_device(K, trace=trace, stream=stream.cuda_stream)
                b.record(stream)
                torch.cuda.synchronize()
                res[f"{order}/{name}"] = {"trace": trace.cpu().numpy(), "ms_per_iter": a.elapsed_time(b) / K}
                s.close()
        best = max(float(v["trace"][-1]) for v in res.values())
        target = best - TTB_TOL * abs(best)
        row = {}
        for key, v in res.items():
            row[key] = {"bound": float(v["trace"][-1]), "iters_to_target": first_within(v["trace"], target),
                        "ms_per_iter": v["ms_per_iter"]}
        out[CONFIG_NAMES[k]] = {"best_bound": best, "target": target, "variants": row}
    return out


def run_split(args, stream) -> dict:
    """Sub-BDDs with copy-arc duals (Sec. 6) on the wide, deep tomography BDDs (64x64 image, 3
    levels; projections up to 128 layers and 97 nodes wide): the whole BDDs; the variable order
    cut into k intervals of similar node counts, k = 4, 32, 128; and the depth split into pieces of
    at most D = 64, 32, 16, 8 layers.  Per variant: device ms per iteration and arcs/s of the
    stated workload (zero unaries), the sweep kernels' ms, and on the tie-break variant (unaries
    N(0, 0.01)) the iterations and ms until the bound is within 1e-3 (relative) of the oracle's
    unsplit bound after --split-ttb-iters iterations, out of three times as many."""
    import torch

    import oracle
    from instances import tomography
    from oracle import Oracle
    from paper_2009_00481_gb300 import Solver

    K, KT = args.split_iters, args.split_ttb_iters
    work = config(2)
    tie = tomography(side=64, seed=0, unary_sigma=0.01)
    oracle.build()
    t0 = time.perf_counter()
    lb_ref = float(Oracle(tie).run_parallel(KT, omega=0.5)[-1])
    oracle_s = time.perf_counter() - t0
    target = ttb_target(lb_ref)
    out = {"workload": CONFIG_NAMES[2], "tie_break_workload": "tomography_64x64x3 with N(0, 0.01) unaries",
           "iterations_timed": K, "gamma": 0.5, "oracle_unsplit_bound": lb_ref,
           "oracle_iterations": KT, "oracle_s": oracle_s, "target": target, "variants": {}}
    trace = torch.zeros(max(K, 3 * KT), dtype=torch.float64, device="cuda")
    variants = [("whole", {})] + [(f"intervals_{k}", {"split": k}) for k in (4, 32, 128)] + \
        [(f"depth_{d}", {"split_depth": d}) for d in (64, 32, 16, 8)]
    for label, kw in variants:
        row = {}
        for name, inst, iters in (("stated", work, K), ("tie_break", tie, 3 * KT)):
            s = Solver(inst, omega=0.5, stream=stream.cuda_stream, **kw)
            s.iterate_device(min(iters, 16), trace=trace, stream=stream.cuda_stream)  # warm-up (graphs)
            s.set_costs(inst.c)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            s.iterate_device(iters, trace=trace, stream=stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms_it = a.elapsed_time(b) / iters
            tr = trace[:iters].cpu().numpy()
            if name == "stated":
                s.set_costs(inst.c)
                kms = s.iterate_profiled(min(iters, 50)) / min(iters, 50)
                row.update({"pieces": s.nb, "cuts": s.n_cuts, "copy_pairs": s.npairs,
                            "max_depth": s.max_depth, "ms_per_iter": ms_it,
                            "arcs_per_s": 2 * s.N / (ms_it / 1e3),
                            "kernel_ms_per_iter": {"fwd": float(kms[0]), "pending_and_cut": float(kms[1]),
                                                   "bwd": float(kms[2]),
                                                   "pending_bound_and_cut": float(kms[3])}})
            else:
                kh = first_within(tr, target)
                row.update({"tie_break_ms_per_iter": ms_it, "tie_break_bound": float(tr[-1]),
                            "iters_to_target": kh, "ms_to_target": ms_it * kh if kh else None})
            s.close()
        out["variants"][label] = row
    return out


# ------------------------------------------------------------------------------------------
# the reference arm: the FP64 oracle on the host cores
# ------------------------------------------------------------------------------------------
def reference_sample(count: int):
    """Batch instances the reference arm cycles through: the ones below 400k coefficients (a
    step of the single-threaded oracle then takes a second or less)."""
    return [s_ for s_ in range(count) if batch_nnz(s_) < 400_000]


def reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    from oracle import Oracle
    oracle.build()
    k = args.config
    iters = args.iters or CONFIG_ITERS[k]
    if k == 4:
        from instances import potts_batch_member
        members = reference_sample(args.batch_count)
        insts = [potts_batch_member(s_) for s_ in members]
        sample = (f"each step: the oracle's {iters} iterations on one instance of the batch, cycling through "
                  f"the {len(members)} instances below 400k coefficients ({members}), FP64 single thread")
    else:
        insts = [config(k)]
        sample = f"full {CONFIG_NAMES[k]} instance, {iters} iterations per step, FP64 single thread"
    orcs = [Oracle(i) for i in insts]
    arcs, secs = 0, 0.0
    tr = None
    for step in range(args.warmup + args.steps):
        o = orcs[step % len(orcs)]
        o.reset()
        t0 = time.perf_counter()
        tr = o.run_parallel(iters, omega=0.5)
        sec = time.perf_counter() - t0
        if step >= args.warmup:
            arcs += 2 * o.N * iters
            secs += sec
    value = arcs / secs
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": CONFIG_NAMES[k], "iterations_per_step": iters, "parallelism": "single"},
           "bound_last_step": float(tr[-1]),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference(args)
        return
    if args.split_only or args.variants_only:
        import torch
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        key = "sub_bdds" if args.split_only else "order_and_averaging"
        res = run_split(args, stream) if args.split_only else run_variants(args, stream)
        print(json.dumps({"metric": METRIC, key: res}), flush=True)
        return
    if args.smoothed_only:
        import torch
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        print(json.dumps({"metric": METRIC, "smoothed": run_smoothed(args, torch, stream, None, reps=args.steps)}),
              flush=True)
        return
    if args.config == 4:
        run_batch(args)
    else:
        run_single(args)


if __name__ == "__main__":
    main()
