#!/usr/bin/env python
"""Benchmark of the dual iteration (forward sweep, reduction, backward sweep, reduction with the
FP64 bound) on the sparse graph matching workload (300x300 points, 10 candidates each, 20000
linearised quadratic pairs; 500 iterations per step).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config C]

A step is one full run of the workload's iteration count from the initial multipliers (the
solver is restarted before each step, outside the timed region; L2 is flushed by a 256 MiB
write before each step).  value = BDD arcs processed per second (2 x nodes x iterations per
step, all ranks) from CUDA events on the launching stream.  `--impl reference` times the FP64
oracle on the host cores instead (rank 0 only).
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--iters", type=int, default=0, help="iterations per step (default: the workload's)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", type=int, default=1, help="1 per-phase graphs (default), 0 persistent kernel")
    ap.add_argument("--staging", type=int, default=-1,
                    help="warp-tile staging of the update sweeps: -1 autotuned (default), 0 bulk-copy ring, "
                         "1 8-layer cp.async windows, 2 the same double-buffered")
    ap.add_argument("--batch-count", type=int, default=256, help="instances in the batch workload")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--batch-warmup", type=int, default=2)
    ap.add_argument("--no-plain", action="store_true", help="batch workload: skip the one-solver-per-instance loop")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch workload part of the default line")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation part of the default line")
    ap.add_argument("--diff-steps", type=int, default=3)
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the variable-order / averaging comparison of the default line")
    ap.add_argument("--variant-iters", type=int, default=300)
    ap.add_argument("--variants-only", action="store_true", help="print only the order / averaging comparison")
    ap.add_argument("--no-split", action="store_true", help="skip the sub-BDD (interval split) comparison")
    ap.add_argument("--split-only", action="store_true", help="print only the sub-BDD comparison")
    ap.add_argument("--split-iters", type=int, default=200, help="timed iterations per sub-BDD variant")
    ap.add_argument("--split-ttb-iters", type=int, default=300,
                    help="oracle iterations giving the sub-BDD comparison's target bound (the GPU runs 3x)")
    return ap.parse_args()


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


def algorithmic_bytes(kind: str, N: int, O: int, n: int, nb: int) -> int:
    if kind in ("fwd", "bwd"):
        # per node: lo/hi 8 B, fm 4 B, bm 4 B; per occurrence: node offset 4, lambda read+write
        # 8, share 4, slot 4, difference write 4; per BDD: depth (+ root value on the backward
        # sweep)
        return 16 * N + 24 * O + (4 if kind == "fwd" else 8) * nb
    if kind == "pending":
        # per variable: slot range 4, P write 4; per slot: difference 4, occurrence id 4,
        # share write 4
        return 8 * n + 12 * O
    if kind == "pending_bound":
        return algorithmic_bytes("pending", N, O, n, nb) + 4 * nb
    if kind == "iteration":
        return sum(algorithmic_bytes(k, N, O, n, nb) for k in ("fwd", "pending", "bwd", "pending_bound"))
    raise ValueError(kind)


STAGING = {0: "bulk-copy ring, 4-layer windows", 1: "8-layer cp.async windows",
           2: "double-buffered 8-layer cp.async windows"}


def staging_of(s) -> dict:
    """Warp-tile staging the solver's autotuner chose for each update sweep."""
    return {"forward": STAGING[s.staging & 3], "backward": STAGING[(s.staging >> 2) & 3]}


def sweep_kernel_name(kind: str, s) -> str:
    st = staging_of(s)
    return {"fwd": f"sweep_kernel<forward, update> ({st['forward']})",
            "bwd": f"sweep_kernel<backward, update> ({st['backward']})",
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
    """Whole-job throughput of `world` independent replicas: all ranks' units over the slowest
    rank's time."""
    return world * units_per_step_per_rank / (ms_max / 1e3)


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
# CPU side: the oracle (bounded sample) -- reference bound for time-to-bound, CPU baseline
# ------------------------------------------------------------------------------------------
def oracle_run(inst, iters, min_seconds=0.0, max_runs=50):
    """Runs the oracle's deferred-averaging schedule from the initial multipliers `iters`
    iterations, repeated until min_seconds have passed.  Returns (final bound, seconds per run,
    runs)."""
    import oracle
    oracle.build()
    from oracle import Oracle
    o = Oracle(inst)
    times, lb = [], None
    while True:
        o.reset()
        t0 = time.perf_counter()
        tr = o.run_parallel(iters, omega=0.5)
        times.append(time.perf_counter() - t0)
        lb = float(tr[-1])
        if sum(times) >= min_seconds or len(times) >= max_runs:
            break
    return lb, float(np.mean(times)), len(times), o.N


def ours(args):
    import torch
    import torch.distributed as dist

    from paper_2009_00481_gb300 import Solver

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if world > 1:
            dist.barrier()

    k = args.config
    iters = args.iters or CONFIG_ITERS[k]
    inst = config(k)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = Solver(inst, omega=0.5, stream=stream.cuda_stream, schedule=args.schedule, staging=args.staging)
    arcs_per_step = 2 * s.N * iters
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    trace = torch.zeros(iters, dtype=torch.float64, device="cuda")

    def step():
        s.iterate_device(iters, trace=trace, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        s.set_costs(inst.c)
        step()
    torch.cuda.synchronize()

    # reference bound for time-to-bound (oracle, rank 0), and the CPU baseline
    cpu = None
    lb_ref = None
    if rank == 0:
        min_s = 0.0 if (args.no_cpu_baseline or world > 1) else 10.0
        lb_ref, sec, runs, _ = oracle_run(inst, iters, min_seconds=min_s, max_runs=20)
        if world == 1 and not args.no_cpu_baseline:
            cpu = {"value": arcs_per_step / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"full {CONFIG_NAMES[k]} instance, {iters} iterations from the initial "
                             f"multipliers, {runs} run(s), FP64 single thread"}

    sampler = ClockSampler(local_rank)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        s.set_costs(inst.c)  # restart from the initial multipliers (host-synchronous, untimed)
        flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = max_over_ranks(float(np.mean(step_ms)), world, device="cuda")
    value = replica_throughput(arcs_per_step, ms, world)
    tr = trace.cpu().numpy()

    # roofline of the dominant kernel.  Persistent schedule: the one iteration kernel, timed by
    # the step's events (one launch per step).  Per-phase schedule: the slowest of the per-phase
    # kernels, timed kernel by kernel with events.  Both report the per-phase breakdown.
    s.set_costs(inst.c)
    kms = s.iterate_profiled(iters)
    kinds = ["fwd", "pending", "bwd", "pending_bound"]
    peak, peak_kind = measured_peaks()
    iter_bytes = algorithmic_bytes("iteration", s.N, s.O, s.n, s.nb)
    if s.schedule == 0:
        kernel_name = "iterate_kernel (persistent, all iterations of a step)"
        abytes = iter_bytes * iters
        per_launch_ms = ms
        launches = args.steps
    else:
        dom = int(np.argmax(kms))
        kernel_name = sweep_kernel_name(kinds[dom], s)
        abytes = algorithmic_bytes(kinds[dom], s.N, s.O, s.n, s.nb)
        per_launch_ms = kms[dom] / iters
        launches = args.steps * graph_launches(iters)
    achieved = abytes / (per_launch_ms / 1e3) / 1e9

    # end to end through the C ABI with host buffers: build (host compile + upload), iterate,
    # read back the bound, multipliers and min-marginals
    e2e = None
    if args.e2e_steps > 0:
        times = []
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = Solver(inst, omega=0.5, schedule=args.schedule, staging=args.staging)
            s2.iterate(iters, lam=True, mm=True)
            s2.close()
            times.append(time.perf_counter() - t0)
        h2d = (inst.row_ptr.nbytes + inst.col.nbytes + inst.val.nbytes + inst.b.nbytes
               + inst.sense.nbytes + inst.c.nbytes)
        d2h = 8 + 3 * 4 * inst.nnz
        e2e = {"value": arcs_per_step / float(np.mean(times)), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "includes": "bdd_build (host BDD compile + upload) + "
               "bdd_iterate with bound, lambda and min-marginals to host + bdd_free"}

    batch = None
    if world == 1 and not args.no_batch:
        batch = run_batched(args, stream, plain=False, n_parity=1)
    diff = None
    if world == 1 and not args.no_diff:
        diff = run_differentiation(args, stream)
    variants = None
    if world == 1 and not args.no_variants:
        variants = run_variants(args, stream)
    split = None
    if world == 1 and not args.no_split:
        split = run_split(args, stream)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    ttb = None
    if lb_ref is not None:
        target = lb_ref - TTB_TOL * abs(lb_ref)
        hit = np.nonzero(tr >= target)[0]
        k_hit = int(hit[0]) + 1 if hit.size else None
        ttb = {"oracle_bound": lb_ref, "gpu_bound": float(tr[-1]), "target": target,
               "iterations": k_hit, "ms": ms * k_hit / iters if k_hit else None}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": CONFIG_NAMES[k], "iterations_per_step": iters, "bdds": s.nb,
                   "nodes": s.N, "arcs": 2 * s.N, "occurrences": s.O, "variables": s.n,
                   "omega": 0.5, "l2": "flushed before each step (256 MiB write); working set "
                   f"{iter_bytes / 1e6:.1f} MB per iteration, L2-resident inside a step",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "time_to_bound": ttb,
        "roofline": {"bound": "hbm", "kernel": kernel_name,
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": dram_traffic(CONFIG_NAMES[k], kernel_name, s.N) if s.schedule == 1 else None,
                     "algorithmic_bytes_per_launch": abytes, "launch_ms": per_launch_ms,
                     "per_phase_kernel_ms_per_iteration": {kd: float(v / iters) for kd, v in zip(kinds, kms)}},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "batched": batch,
        "differentiation": diff,
        "order_and_averaging": variants,
        "sub_bdds": split,
        "gpu_launches": launches,
        "schedule": "persistent" if s.schedule == 0 else "per-phase graphs",
        "staging": staging_of(s),
        "clocks": clocks,
        "wall_s": wall,
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batched(args, stream, plain: bool, n_parity: int) -> dict:
    """The batch of 256 uneven Potts instances packed into one solver (one launch chain for all
    instances): throughput, the roofline of the dominant kernel, per-instance parity with the
    oracle on a bounded sample, and optionally the plain form (one solver per instance, solved
    one after another) for comparison."""
    import torch

    from instances import potts_batch, potts_batch_member
    from paper_2009_00481_gb300 import Solver

    iters = CONFIG_ITERS[4] if args.config != 4 or not args.iters else args.iters
    count = args.batch_count
    t0 = time.perf_counter()
    inst = potts_batch(count)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    s = Solver(inst, omega=0.5, stream=stream.cuda_stream, schedule=args.schedule, staging=args.staging)
    build_s = time.perf_counter() - t0
    arcs_per_step = 2 * s.N * iters
    trace = torch.zeros(iters, dtype=torch.float64, device="cuda")

    def step():
        s.iterate_device(iters, trace=trace, stream=stream.cuda_stream)

    warmup = args.batch_warmup
    steps = args.batch_steps
    for _ in range(warmup):
        s.set_costs(inst.c)
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        s.set_costs(inst.c)
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    bounds = s.bound_parts(inst.row_parts, inst.var_parts)

    # per-instance time to a bound within 1e-3 of the instance's bound after the step's
    # iterations: an untimed rerun one iteration at a time, every instance's FP64 bound after
    # each (the reference bounds are the packed solve's own, checked against the oracle on the
    # sampled instances below)
    s.set_costs(inst.c)
    traj = np.zeros((iters, count))
    for it in range(iters):
        s.iterate_device(1, stream=stream.cuda_stream)
        traj[it] = s.bound_parts(inst.row_parts, inst.var_parts)
    final = traj[-1]
    hit = traj >= (final - TTB_TOL * np.abs(final))[None, :]
    first = np.argmax(hit, axis=0) + 1  # hit[-1] is always true
    ms_iter = ms / iters
    per_instance = {"reference": "each instance's bound after the step's iterations (packed solve)",
                    "tolerance": TTB_TOL, "instances": count,
                    "iterations": {"median": float(np.median(first)), "p90": float(np.percentile(first, 90)),
                                   "max": int(first.max()), "min": int(first.min())},
                    "ms": {"median": float(np.median(first)) * ms_iter, "p90": float(np.percentile(first, 90)) * ms_iter,
                           "max": float(first.max()) * ms_iter},
                    "final_matches_timed_run": bool(np.array_equal(final, bounds))}

    # per-phase kernels, timed one by one, for the roofline of the dominant kernel
    s.set_costs(inst.c)
    kms = s.iterate_profiled(iters)
    kinds = ["fwd", "pending", "bwd", "pending_bound"]
    dom = int(np.argmax(kms))
    peak, peak_kind = measured_peaks()
    abytes = algorithmic_bytes(kinds[dom], s.N, s.O, s.n, s.nb)
    per_launch_ms = kms[dom] / iters
    achieved = abytes / (per_launch_ms / 1e3) / 1e9
    iter_bytes = algorithmic_bytes("iteration", s.N, s.O, s.n, s.nb)
    iter_ms = float(kms.sum() / iters)

    # the oracle on a bounded sample of every 32nd instance (the smallest ones): per-instance
    # parity and the CPU baseline
    import oracle
    oracle.build()
    from oracle import Oracle
    every = list(range(0, count, max(1, count // 8)))
    sizes = [potts_batch_member(idx).nnz for idx in every]
    sample = sorted(every[t] for t in np.argsort(sizes, kind="stable")[:n_parity])
    cpu_arcs, cpu_s, parity = 0, 0.0, []
    for idx in sample:
        o = Oracle(potts_batch_member(idx))
        t0 = time.perf_counter()
        tr = o.run_parallel(iters, omega=0.5)
        cpu_s += time.perf_counter() - t0
        cpu_arcs += 2 * o.N * iters
        want, got = float(tr[-1]), float(bounds[idx])
        parity.append({"instance": idx, "oracle": want, "gpu": got,
                       "rel_err": abs(got - want) / max(1.0, abs(want))})

    plain_d = None
    if plain:
        solvers = [Solver(potts_batch_member(idx), omega=0.5, stream=stream.cuda_stream, schedule=args.schedule)
                   for idx in range(count)]
        for t in solvers:
            t.iterate_device(2, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in solvers:
            t.iterate_device(iters, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        plain_d = {"value": arcs_per_step / (pms / 1e3), "unit": UNIT, "ms": pms,
                   "form": f"{count} solvers, one per instance, iterated one after another"}
        for t in solvers:
            t.close()
    s.close()
    return {
        "value": arcs_per_step / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
        "config": {"workload": CONFIG_NAMES[4], "instances": count, "iterations_per_step": iters,
                   "bdds": s.nb, "nodes": s.N, "arcs": 2 * s.N, "occurrences": s.O, "variables": s.n,
                   "omega": 0.5, "device_bytes": s.device_bytes,
                   "l2": f"inputs larger than L2: {iter_bytes / 1e9:.2f} GB moved per iteration",
                   "generate_s": gen_s, "build_s": build_s},
        "roofline": {"bound": "hbm", "kernel": sweep_kernel_name(kinds[dom], s),
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": dram_traffic(CONFIG_NAMES[4], sweep_kernel_name(kinds[dom], s), s.N), "algorithmic_bytes_per_launch": abytes,
                     "launch_ms": per_launch_ms,
                     "iteration": {"algorithmic_bytes": iter_bytes, "ms": iter_ms,
                                   "achieved_gbs": iter_bytes / (iter_ms / 1e3) / 1e9,
                                   "frac": iter_bytes / (iter_ms / 1e3) / 1e9 / peak},
                     "per_phase_kernel_ms_per_iteration": {kd: float(v / iters) for kd, v in zip(kinds, kms)}},
        "parity_sampled_instances": parity,
        "time_to_bound_per_instance": per_instance,
        "cpu_baseline": {"value": cpu_arcs / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"instances {sample} of the batch, {iters} iterations each, FP64 single thread"},
        "plain_loop": plain_d,
        "gpu_launches": steps * graph_launches(iters),
        "schedule": "persistent" if s.schedule == 0 else "per-phase graphs",
        "staging": staging_of(s),
        "clocks": clocks,
    }


def run_differentiation(args, stream) -> dict:
    """The differentiation workload (cell-tracking-shaped flow ILP, 50 frames x 200 detections):
    K = 50 smoothed iterations (tau = 0.1) forward, and forward plus the adjoint giving
    d(bound)/dc, against K plain iterations on the same instance; smoothed-bound parity with the
    oracle and a central-difference gradient check on the 5-frame x 20-detection slice."""
    import torch

    from instances import tracking
    from paper_2009_00481_gb300 import Solver, binding

    inst = config(3)
    K, alpha = CONFIG_ITERS[3], 0.1
    reps = args.diff_steps
    plain = Solver(inst, omega=0.5, stream=stream.cuda_stream)
    smooth = Solver(inst, omega=0.5, stream=stream.cuda_stream, alpha=alpha)
    arcs = 2 * plain.N * K
    c = torch.tensor(inst.c, device="cuda")
    bound = torch.zeros((), dtype=torch.float64, device="cuda")
    gbound = torch.ones((), dtype=torch.float64, device="cuda")
    grad = torch.zeros(inst.n, dtype=torch.float32, device="cuda")
    trace = torch.zeros(K, dtype=torch.float64, device="cuda")
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

    def plain_step():
        plain.set_costs(inst.c)
        plain.iterate_device(K, trace=trace, stream=sp)

    ms_plain = timed(plain_step)
    plain_bound = float(trace[-1].item())
    ms_fwd = timed(lambda: binding.bdd_smooth_forward(smooth.h, K, c.data_ptr(), bound.data_ptr(), sp))

    def fwd_bwd():
        gen = binding.bdd_smooth_forward(smooth.h, K, c.data_ptr(), bound.data_ptr(), sp)
        binding.bdd_smooth_backward(smooth.h, gen, gbound.data_ptr(), grad.data_ptr(), sp)

    ms_fb = timed(fwd_bwd)
    smooth_bound = float(bound.item())

    import oracle
    oracle.build()
    from oracle import Oracle
    o = Oracle(inst)
    o.set_alpha(alpha)
    want = float(o.run_parallel(K, omega=0.5)[-1])

    # gradient check on the slice: 8 coordinates, FP64 central differences of the oracle
    import copy
    sl = tracking(frames=5, dets=20, seed=0)
    ss = Solver(sl, omega=0.5, stream=sp, alpha=alpha)
    csl = torch.tensor(sl.c, device="cuda")
    gsl = torch.zeros(sl.n, dtype=torch.float32, device="cuda")
    gen = binding.bdd_smooth_forward(ss.h, K, csl.data_ptr(), bound.data_ptr(), sp)
    binding.bdd_smooth_backward(ss.h, gen, gbound.data_ptr(), gsl.data_ptr(), sp)
    g = gsl.cpu().numpy().astype(np.float64)

    def ob(cv):
        j = copy.copy(sl)
        j.c = cv
        oo = Oracle(j)
        oo.set_alpha(alpha)
        return float(oo.run_parallel(K, omega=0.5)[-1])

    idx = np.random.default_rng(0).choice(sl.n, size=8, replace=False)
    h = 1e-4
    c0 = sl.c.astype(np.float64)
    fd = []
    for i in idx:
        cp, cm = c0.copy(), c0.copy()
        cp[i] += h
        cm[i] -= h
        fd.append((ob(cp) - ob(cm)) / (2 * h))
    fd = np.asarray(fd)
    grad_err = float(np.abs(g[idx] - fd).max() / max(1.0, np.abs(fd).max()))
    for t in (plain, smooth, ss):
        t.close()
    return {
        "workload": CONFIG_NAMES[3], "iterations": K, "tau": alpha, "nodes": arcs // (2 * K),
        "plain": {"value": arcs / (ms_plain / 1e3), "unit": UNIT, "ms": ms_plain, "bound": plain_bound},
        "smoothed_forward": {"value": arcs / (ms_fwd / 1e3), "unit": UNIT, "ms": ms_fwd, "bound": smooth_bound,
                             "oracle_bound": want, "rel_err": abs(smooth_bound - want) / max(1.0, abs(want))},
        "smoothed_forward_backward": {"value": arcs / (ms_fb / 1e3), "unit": UNIT, "ms": ms_fb,
                                      "note": "K smoothed iterations with per-sweep checkpoints, then the "
                                              "adjoint pass (recomputation + adjoint kernels) giving d(bound)/dc"},
        "gradient_check": {"slice": "tracking 5 frames x 20 detections", "coordinates": 8,
                           "max_err_rel_to_max_grad": grad_err, "reference": "FP64 central differences of the oracle"},
    }


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
            hit = np.nonzero(v["trace"] >= target)[0]
            row[key] = {"bound": float(v["trace"][-1]), "iters_to_target": int(hit[0]) + 1 if hit.size else None,
                        "ms_per_iter": v["ms_per_iter"]}
        out[CONFIG_NAMES[k]] = {"best_bound": best, "target": target, "variants": row}
    return out


def run_split(args, stream) -> dict:
    """Sub-BDDs with copy-arc duals (Sec. 6) on the wide, deep tomography BDDs (64x64 image, 3
    levels; projections up to 128 layers and 97 nodes wide): the whole BDDs; the variable order
    cut into k intervals of similar node counts, k = 4, 32, 128 (a row projection covers 192
    consecutive variables, so only many intervals cut all of them); and the depth split into
    pieces of at most D = 64, 32, 16, 8 layers.  Per variant: device ms per iteration
    and arcs/s of the stated workload (zero unaries), the forward / backward sweep kernels' ms,
    and on the tie-break variant (unaries N(0, 0.01)) the iterations and ms until the bound is
    within 1e-3 (relative) of the oracle's unsplit bound after --split-ttb-iters iterations, out
    of three times as many (a split relaxes the rows until the copy duals agree, so it may need
    more iterations)."""
    import torch

    from paper_2009_00481_gb300 import Solver
    from instances import tomography

    K, KT = args.split_iters, args.split_ttb_iters
    work = config(2)
    tie = tomography(side=64, seed=0, unary_sigma=0.01)
    t0 = time.perf_counter()
    lb_ref, _, _, _ = oracle_run(tie, KT)
    oracle_s = time.perf_counter() - t0
    target = lb_ref - TTB_TOL * abs(lb_ref)
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
                hit = np.nonzero(tr >= target)[0]
                kh = int(hit[0]) + 1 if hit.size else None
                row.update({"tie_break_ms_per_iter": ms_it, "tie_break_bound": float(tr[-1]),
                            "iters_to_target": kh, "ms_to_target": ms_it * kh if kh else None})
            s.close()
        out["variants"][label] = row
    return out


def batched(args):
    """`--config 4`: the batch workload as the bench line."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    b = run_batched(args, stream, plain=not args.no_plain, n_parity=3)
    out = {"metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": 1, "steps": b["steps"],
           "warmup": b["warmup"], "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": dict(b["config"], parallelism="single")}
    out.update({k: b[k] for k in ("roofline", "parity_sampled_instances", "cpu_baseline", "plain_loop",
                                  "gpu_launches", "schedule", "clocks")})
    print(json.dumps(out), flush=True)


def reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    k = args.config
    iters = args.iters or CONFIG_ITERS[k]
    inst = config(k)
    import oracle
    oracle.build()
    from oracle import Oracle
    o = Oracle(inst)
    arcs_per_step = 2 * o.N * iters

    def step():
        o.reset()
        return o.run_parallel(iters, omega=0.5)

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        tr = step()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = arcs_per_step / (ms / 1e3)
    sample = (f"full {CONFIG_NAMES[k]} instance, {iters} iterations per step from the initial "
              "multipliers, FP64 single thread")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": CONFIG_NAMES[k], "iterations_per_step": iters, "nodes": o.N,
                      "arcs": 2 * o.N, "parallelism": "single"},
           "bound": float(tr[-1]),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference(args)
    elif args.config == 4:
        batched(args)
    elif args.split_only:
        import torch
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        print(json.dumps({"metric": METRIC, "sub_bdds": run_split(args, stream)}), flush=True)
    elif args.variants_only:
        import torch
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        print(json.dumps({"metric": METRIC, "order_and_averaging": run_variants(args, stream)}), flush=True)
    elif args.config == 3:
        import torch
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        print(json.dumps({"metric": METRIC, "differentiation": run_differentiation(args, stream)}), flush=True)
    else:
        ours(args)


if __name__ == "__main__":
    main()
