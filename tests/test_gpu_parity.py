"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the same seeded
inputs.

Tolerances (relative with a floor of 1: |a - b| <= tol * max(1, |a|, |b|)):
  - BDD node / arc arrays read back from the device: bit-exact;
  - min-marginals for the same FP32 multipliers: 1e-5 (FP32 path sums of at most a few hundred
    terms of magnitude <= the bound scale);
  - lower bound after 100 iterations of the deferred-averaging schedule (same omega): 1e-4;
  - the device bound trace never drops by more than 1e-5 * |bound|.
"""
from __future__ import annotations

import numpy as np
import pytest

from instances import (SENSE_LE, config, potts_mrf, random_ilp, sparse_matching, tomography,
                       tracking)
from instances.generators import _from_rows
from oracle import Oracle

pytestmark = pytest.mark.gpu

MM_TOL = 1e-5
LB_TOL = 1e-4
MONO_TOL = 1e-5


def close(a, b, tol):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    fin = np.isfinite(a) & np.isfinite(b)
    assert np.array_equal(np.isfinite(a), np.isfinite(b)), "infinite entries differ"
    assert np.array_equal(np.sign(a[~fin]), np.sign(b[~fin]))
    err = np.abs(a[fin] - b[fin]) / np.maximum(1.0, np.maximum(np.abs(a[fin]), np.abs(b[fin])))
    assert err.size == 0 or err.max() <= tol, f"max rel err {err.max():.3e} > {tol:.1e}"


@pytest.fixture(scope="module")
def lib(cuda_lib):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return cuda_lib


def solver(inst, **kw):
    from paper_2009_00481_gb300 import Solver
    return Solver(inst, **kw)


CASES = {
    "potts_20x20x3": lambda: config(0),
    "matching_300x300": lambda: config(1),
    "matching_small": lambda: sparse_matching(n_left=60, n_right=50, k=6, n_pairs=800, seed=3),
    "tomography_16": lambda: tomography(side=16, seed=1, unary_sigma=0.05),
    "tracking_10x40": lambda: tracking(frames=10, dets=40, seed=1),
    "random_wide": lambda: random_ilp(n=60, m=40, max_row_vars=16, seed=11, coef=3),
}


# ------------------------------------------------------------------------------------------
# structure
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", sorted(CASES))
def test_device_slabs_bit_exact(lib, name):
    inst = CASES[name]()
    want = Oracle(inst).canonical()
    got = solver(inst).canonical()
    for key in ["bdd_row", "bdd_depth", "occ_var", "occ_csr", "occ_width", "lo", "hi"]:
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)


def test_device_slabs_full_tomography(lib):
    inst = config(2)
    want = Oracle(inst).canonical()
    got = solver(inst).canonical()
    for key in ["bdd_row", "bdd_depth", "occ_var", "occ_csr", "occ_width", "lo", "hi"]:
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)


# ------------------------------------------------------------------------------------------
# min-marginals for the same multipliers (standalone pass)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", sorted(CASES))
def test_min_marginals_same_lambda(lib, name):
    inst = CASES[name]()
    rng = np.random.default_rng(5)
    lam = rng.normal(0, 1, size=inst.nnz).astype(np.float32)
    lam[inst.val == 0] = 0
    s = solver(inst)
    s.set_state(lam)
    lb, lam_out, m0, m1 = s.iterate(0, lam=True, mm=True)
    o = Oracle(inst)
    o.set_state(lam.astype(np.float64))
    e0, e1 = o.min_marginals(fold=True)
    close(m0, e0, MM_TOL)
    close(m1, e1, MM_TOL)
    np.testing.assert_array_equal(lam_out, lam)  # no pending share: lambda unchanged
    close([lb], [o.bound()], MM_TOL)


def _wide_rows_instance():
    """A 300-variable cardinality row (layers up to 150 nodes wide: block tiles with several nodes
    per thread) plus narrow rows of every warp team size."""
    rng = np.random.default_rng(3)
    rows = [(np.arange(300), np.ones(300), 149, SENSE_LE)]
    for k in [2, 3, 5, 9, 17, 33, 40]:
        cols = np.sort(rng.choice(300, size=k, replace=False))
        rows.append((cols, np.ones(k), k // 2, SENSE_LE))
    c = rng.normal(size=300).astype(np.float32)
    return _from_rows("wide", 300, rows, c)


@pytest.mark.parametrize("which", ["tomography_64x64", "wide_rows"])
def test_min_marginals_same_lambda_block_tiles(lib, which):
    """Same-multiplier min-marginals element by element on the two block-tile paths: the
    one-node-per-thread path (full 64x64 tomography: projection layers of 33..97 nodes) and the
    general path (a row whose layers exceed 128 nodes)."""
    inst = config(2) if which == "tomography_64x64" else _wide_rows_instance()
    s = solver(inst)
    o = Oracle(inst)
    if which == "tomography_64x64":
        assert 32 < o.max_width <= 128
    else:
        assert o.max_width > 128
    assert s.block_tiles >= 1
    rng = np.random.default_rng(12)
    lam = rng.normal(0, 1, size=inst.nnz).astype(np.float32)
    lam[inst.val == 0] = 0
    P = rng.normal(0, 0.5, size=inst.n).astype(np.float32)
    s.set_state(lam, P)
    lb, lam_out, m0, m1 = s.iterate(0, lam=True, mm=True)
    o.set_state(lam.astype(np.float64), P.astype(np.float64))
    e0, e1 = o.min_marginals(fold=True)
    close(m0, e0, MM_TOL)
    close(m1, e1, MM_TOL)
    close(lam_out, o.lam(fold=True), 1e-6)
    close([lb], [o.bound()], MM_TOL)


def test_min_marginals_with_pending_share(lib):
    """Outputs fold the pending share P_i/|J_i| into lambda before the pass."""
    inst = CASES["matching_small"]()
    rng = np.random.default_rng(8)
    lam = rng.normal(0, 1, size=inst.nnz).astype(np.float32)
    P = rng.normal(0, 0.5, size=inst.n).astype(np.float32)
    s = solver(inst)
    s.set_state(lam, P)
    lb, lam_out, m0, m1 = s.iterate(0, lam=True, mm=True)
    o = Oracle(inst)
    o.set_state(lam.astype(np.float64), P.astype(np.float64))
    close(lam_out, o.lam(fold=True), 1e-6)
    e0, e1 = o.min_marginals(fold=True)
    close(m0, e0, MM_TOL)
    close(m1, e1, MM_TOL)
    close([lb], [o.bound()], MM_TOL)


# ------------------------------------------------------------------------------------------
# iterations: bound trace parity with the oracle's schedule
# ------------------------------------------------------------------------------------------

def _trace(s, iters):
    import torch
    tr = torch.zeros(iters, dtype=torch.float64, device="cuda")
    s.iterate_device(iters, trace=tr)
    torch.cuda.synchronize()
    return tr.cpu().numpy()


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("omega", [0.5, 1.0])
@pytest.mark.parametrize("name", sorted(CASES))
def test_bound_trace_parity(lib, name, omega, schedule):
    inst = CASES[name]()
    iters = 100
    want = Oracle(inst).run_parallel(iters, omega=omega)
    got = _trace(solver(inst, omega=omega, schedule=schedule), iters)
    close(got, want, LB_TOL)  # every iterate
    scale = np.maximum(1.0, np.abs(got[1:]))
    assert np.all(np.diff(got) >= -MONO_TOL * scale), "device bound decreased"


@pytest.mark.parametrize("k", [1, 3])
def test_bound_parity_workloads_full(lib, k):
    """Matching 300x300 at its 500 iterations; tracking 50x200 at 50 iterations."""
    inst = config(k)
    iters = {1: 500, 3: 50}[k]
    want = Oracle(inst).run_parallel(iters, omega=0.5)
    got = _trace(solver(inst), iters)
    close(got, want, LB_TOL)  # every iterate


def test_bound_parity_tomography_full(lib):
    """64x64 tomography with unary tie-break costs (the all-zero-cost workload sits at a fixed
    point of the non-smooth method), 100 iterations."""
    inst = tomography(side=64, seed=0, unary_sigma=0.01)
    want = Oracle(inst).run_parallel(100, omega=0.5)
    got = _trace(solver(inst), 100)
    close(got, want, LB_TOL)  # every iterate


def test_zero_cost_tomography_stays_at_zero(lib):
    inst = config(2)
    got = _trace(solver(inst), 20)
    assert np.all(got == 0.0)


def test_outputs_after_iterations(lib):
    """lambda folded and min-marginals after 100 iterations match the oracle's; the folded
    multipliers of each variable sum to c_i."""
    inst = config(0)
    s = solver(inst)
    lb, lam, m0, m1 = s.iterate(100, lam=True, mm=True)
    o = Oracle(inst)
    tr = o.run_parallel(100, omega=0.5)
    close([lb], [tr[-1]], LB_TOL)
    close(lam, o.lam(fold=True), 2e-4)
    e0, e1 = o.min_marginals(fold=True)
    close(m0, e0, 5e-4)
    close(m1, e1, 5e-4)
    sums = np.zeros(inst.n)
    np.add.at(sums, inst.col, lam.astype(np.float64))
    close(sums, inst.c, 1e-5)


# ------------------------------------------------------------------------------------------
# determinism, state and outputs
# ------------------------------------------------------------------------------------------

def test_deterministic(lib):
    inst = config(1)
    a, b = solver(inst), solver(inst)
    ta, tb = _trace(a, 60), _trace(b, 60)
    np.testing.assert_array_equal(ta, tb)
    la, pa = a.get_state()
    lb_, pb = b.get_state()
    np.testing.assert_array_equal(la, lb_)
    np.testing.assert_array_equal(pa, pb)


def test_outputs_leave_state_unchanged(lib):
    inst = CASES["tomography_16"]()
    a, b = solver(inst), solver(inst)
    t1 = _trace(a, 10)
    a.iterate(0, lam=True, mm=True)
    t2 = _trace(a, 10)
    tb = _trace(b, 20)
    np.testing.assert_array_equal(np.concatenate([t1, t2]), tb)


def test_state_roundtrip_resumes_bit_identical(lib):
    inst = CASES["tracking_10x40"]()
    a, b = solver(inst), solver(inst)
    _trace(a, 15)
    lam, P = a.get_state()
    b.set_state(lam, P)
    np.testing.assert_array_equal(_trace(a, 15), _trace(b, 15))


def test_set_costs_restarts(lib):
    inst = config(0)
    s = solver(inst)
    t1 = _trace(s, 20)
    s.set_costs(inst.c)
    np.testing.assert_array_equal(_trace(s, 20), t1)
    c2 = (inst.c * 2).astype(np.float32)
    s.set_costs(c2)
    inst2 = potts_mrf(20, 20, 3, seed=0)
    inst2.c = c2
    close(_trace(s, 20)[-1:], Oracle(inst2).run_parallel(20)[-1:], LB_TOL)


def test_calls_on_different_streams_are_ordered(lib):
    """Device iterations enqueued on a PyTorch stream, then host calls on the solver's own
    stream without any synchronisation in between: the host calls see the finished iterations."""
    import torch
    inst = config(1)
    a, b = solver(inst), solver(inst)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        tr = torch.zeros(40, dtype=torch.float64, device="cuda")
        a.iterate_device(40, trace=tr)
    lb_a, lam_a, _, _ = a.iterate(0, lam=True)
    lb_b, lam_b, _, _ = b.iterate(40, lam=True)
    torch.cuda.synchronize()
    assert lb_a == lb_b
    np.testing.assert_array_equal(lam_a, lam_b)
    np.testing.assert_array_equal(tr.cpu().numpy()[-1], lb_b)


@pytest.mark.parametrize("name", ["potts_20x20x3", "tomography_16", "tracking_10x40", "random_wide"])
def test_schedules_agree(lib, name):
    """The persistent kernel (schedule 0) and the per-phase kernels (schedule 1) run the same
    arithmetic: multipliers and pending sums are bit-identical; bounds differ at most in the
    FP64 summation order."""
    inst = CASES[name]()
    a, b = solver(inst, schedule=0), solver(inst, schedule=1)
    assert a.schedule == 0 and b.schedule == 1
    ta, tb = _trace(a, 30), _trace(b, 30)
    close(ta, tb, 1e-12)
    la, pa = a.get_state()
    lb_, pb = b.get_state()
    np.testing.assert_array_equal(la, lb_)
    np.testing.assert_array_equal(pa, pb)
    # switching schedules mid-run keeps the trajectory
    tb2 = _trace(b, 5)
    c = solver(inst, schedule=0)
    c.set_state(la, pa)
    close(_trace(c, 5), tb2, 1e-12)


def _mixed_degree_instance(seed=5):
    """At-most-one rows of four over variables of three kinds: 6000 of degree about 12 (more than
    4096 above 8, so the heavy-variable threshold is 16), 6000 of degree about 2, and 12 of
    degree about 60 (heavy: one warp each)."""
    rng = np.random.default_rng(seed)
    n = 12000
    need = np.concatenate([np.full(6000, 12), np.full(6000, 2)])
    need[rng.choice(n, size=12, replace=False)] = 60
    pool = np.repeat(np.arange(n), need)
    rng.shuffle(pool)
    rows = []
    for g in range(0, len(pool) - 3, 4):
        cols = np.unique(pool[g:g + 4])
        rows.append((cols, np.ones(len(cols)), 1, SENSE_LE))
    c = rng.standard_normal(n).astype(np.float32)
    return _from_rows("mixed_degrees", n, rows, c)


@pytest.mark.parametrize("averaging", [0, 1])
def test_pending_mixed_degrees_match_persistent(lib, averaging):
    """The per-phase pending pass (one thread per variable with the next slot range loaded
    ahead, variables above the heavy threshold one warp each, the threshold chosen from the
    degree histogram) gives the multipliers and pending sums of the persistent kernel's pass bit
    for bit, with and without SRMP, on a mix of light, medium and heavy variables."""
    inst = _mixed_degree_instance()
    deg = np.bincount(inst.col, minlength=inst.n)
    assert (deg > 16).sum() >= 12 and (deg > 8).sum() > 4096
    a = solver(inst, schedule=0, averaging=averaging)
    b = solver(inst, schedule=1, averaging=averaging)
    assert a.schedule == 0 and b.schedule == 1
    close(_trace(a, 12), _trace(b, 12), 1e-12)
    la, pa = a.get_state()
    lb_, pb = b.get_state()
    np.testing.assert_array_equal(la, lb_)
    np.testing.assert_array_equal(pa, pb)


def test_barrier_timeout_reports_status(lib):
    """A grid-barrier wait limited to one poll gives up; the kernel returns, the host call reports
    BDD_ETIMEOUT, and the device stays usable."""
    from paper_2009_00481_gb300 import BDDError
    from paper_2009_00481_gb300.binding import BDD_ETIMEOUT
    inst = config(1)
    s = solver(inst, schedule=0, spin_limit=1)
    with pytest.raises(BDDError) as e:
        s.iterate(3)
    assert e.value.code == BDD_ETIMEOUT
    s.close()
    ok = solver(inst)
    want = Oracle(inst).run_parallel(5, omega=0.5)
    close(_trace(ok, 5), want, LB_TOL)


def test_host_iterate_matches_device_trace(lib):
    inst = config(0)
    a, b = solver(inst), solver(inst)
    t = _trace(a, 37)
    lb, _, _, _ = b.iterate(37)
    assert lb == t[-1]


@pytest.mark.parametrize("fused", [0, 1])
def test_profiled_iterations_match(lib, fused):
    """Kernel-by-kernel iterations with events reach the state of the graph replays (the fused
    plan has no separate pending pass: its slot reads 0 ms)."""
    inst = config(0)
    a, b = solver(inst, fused_pending=fused), solver(inst, fused_pending=fused)
    ms = a.iterate_profiled(12)
    assert ms.shape == (4,) and ms[0] > 0 and ms[2] > 0 and ms[3] > 0
    assert (ms[1] > 0) if not fused else (ms[1] >= 0)
    lb_a, _, _, _ = a.iterate(0)
    lb_b = _trace(b, 12)[-1]
    close([lb_a], [lb_b], 1e-12)
    la, pa = a.get_state()
    lb_, pb = b.get_state()
    np.testing.assert_array_equal(la, lb_)
    np.testing.assert_array_equal(pa, pb)


@pytest.mark.parametrize("variant", ["plain", "srmp", "smooth", "cm"])
@pytest.mark.parametrize("name", ["potts_20x20x3", "matching_small", "tomography_16", "tracking_10x40",
                                  "random_wide"])
def test_fused_pending_matches_separate_kernels(lib, name, variant):
    """The pending pass fused into the sweeps (last visit of a variable forms P_i) runs the
    separate pending kernel's arithmetic: multipliers and pending sums bit-identical, bounds equal
    up to the FP64 summation order, for 8-iteration graphs plus a ragged tail of 3."""
    inst = CASES[name]()
    kw = {"plain": {}, "srmp": {"averaging": 1}, "smooth": {"alpha": 0.2}, "cm": {"rank": "cm"}}[variant]
    a, b = solver(inst, fused_pending=1, **kw), solver(inst, fused_pending=0, **kw)
    ta, tb = _trace(a, 19), _trace(b, 19)
    close(ta, tb, 1e-12)
    la, pa = a.get_state()
    lb_, pb = b.get_state()
    np.testing.assert_array_equal(la, lb_)
    np.testing.assert_array_equal(pa, pb)
    _, lam_a, m0a, m1a = a.iterate(0, lam=True, mm=True)
    _, lam_b, m0b, m1b = b.iterate(0, lam=True, mm=True)
    np.testing.assert_array_equal(lam_a, lam_b)
    np.testing.assert_array_equal(m0a, m0b)
    np.testing.assert_array_equal(m1a, m1b)


# ------------------------------------------------------------------------------------------
# edge cases
# ------------------------------------------------------------------------------------------

def test_empty_instance(lib):
    inst = _from_rows("empty", 3, [], np.array([1.0, -2.0, -0.5], np.float32))
    s = solver(inst)
    lb, lam, m0, m1 = s.iterate(3, lam=True, mm=True)
    assert lb == pytest.approx(-2.5)


def test_unconstrained_variables_and_single_rows(lib):
    rows = [(np.array([0, 2]), np.array([1, 1]), 1, SENSE_LE), (np.array([2]), np.array([1]), 1, SENSE_LE)]
    inst = _from_rows("u", 4, rows, np.array([-1.0, -3.0, -2.0, 0.5], np.float32))
    want = Oracle(inst).run_parallel(30)
    got = _trace(solver(inst), 30)
    close(got, want, LB_TOL)


def test_wide_block_tiles(lib):
    """A 300-variable cardinality row has layers up to 150 nodes wide (block tiles with several
    nodes per thread), plus narrow rows of every warp team size."""
    inst = _wide_rows_instance()
    o = Oracle(inst)
    assert o.max_width > 128
    s = solver(inst)
    assert s.block_tiles >= 1
    np.testing.assert_array_equal(s.canonical()["lo"], o.canonical()["lo"])
    close(_trace(s, 100), o.run_parallel(100), LB_TOL)


def test_forced_variables(lib):
    """Rows that force variables give +inf min-marginals; the difference is taken as 0."""
    rows = [(np.array([0, 1]), np.array([1, 1]), 2, 0), (np.array([1, 2]), np.array([1, 1]), 1, SENSE_LE),
            (np.array([0, 2, 3]), np.array([1, 1, 1]), 2, SENSE_LE)]
    inst = _from_rows("forced", 4, rows, np.array([1.0, 2.0, -1.0, -0.5], np.float32))
    s = solver(inst)
    lb, lam, m0, m1 = s.iterate(0, mm=True)
    o = Oracle(inst)
    e0, e1 = o.min_marginals(fold=True)
    close(m0, e0, MM_TOL)
    close(m1, e1, MM_TOL)
    close(_trace(s, 20), o.run_parallel(20), LB_TOL)


def test_max_device_bytes(lib):
    from paper_2009_00481_gb300 import BDDError
    from paper_2009_00481_gb300.binding import BDD_ENOMEM
    with pytest.raises(BDDError) as e:
        solver(config(1), max_device_bytes=1 << 16)
    assert e.value.code == BDD_ENOMEM


# ------------------------------------------------------------------------------------------
# batches of independent instances packed into one solver
# ------------------------------------------------------------------------------------------

def _small_batch():
    from instances import potts_batch, potts_batch_member
    kw = dict(side_range=(3, 7), label_range=(2, 4))
    packed = potts_batch(count=5, first_seed=40, **kw)
    members = [potts_batch_member(40 + k, **kw) for k in range(5)]
    return packed, members


def test_batch_part_bounds_match_members(lib):
    """Per-instance bounds of a packed batch equal each instance's own oracle bound, and the
    parts add up to the packed bound."""
    packed, members = _small_batch()
    s = solver(packed)
    tr = _trace(s, 40)
    parts = s.bound_parts(packed.row_parts, packed.var_parts)
    want = [Oracle(m).run_parallel(40, omega=0.5)[-1] for m in members]
    close(parts, want, LB_TOL)
    assert abs(parts.sum() - tr[-1]) <= 1e-9 * max(1.0, abs(tr[-1]))


def test_batch_members_bit_identical_to_separate_solves(lib):
    """Packing independent instances changes no arithmetic: each member's multipliers after
    the packed solve equal those of solving the member alone, bit for bit."""
    packed, members = _small_batch()
    s = solver(packed)
    _trace(s, 25)
    lam, _ = s.get_state()
    off = packed.row_parts
    for k, m in enumerate(members):
        t = solver(m)
        _trace(t, 25)
        lm, _ = t.get_state()
        a, b = int(packed.row_ptr[off[k]]), int(packed.row_ptr[off[k + 1]])
        np.testing.assert_array_equal(lam[a:b], lm)


def test_bound_parts_rejects_bad_offsets(lib):
    from paper_2009_00481_gb300 import BDDError
    packed, _ = _small_batch()
    s = solver(packed)
    with pytest.raises(BDDError):
        s.bound_parts([0, 1], [0, packed.n])


@pytest.mark.parametrize("name", ["potts_20x20x3", "matching_small", "tomography_16", "tracking_10x40",
                                  "random_wide"])
@pytest.mark.parametrize("variant", ["plain", "smooth", "srmp"])
def test_staging_variants_bit_identical(lib, name, variant):
    """The three warp-tile staging variants (bulk-copy ring of 4-layer windows; 8-layer cp.async
    windows, single- and double-buffered) feed the same arithmetic: bound traces, multipliers and
    pending sums bit-identical over graphs of 8 iterations plus a ragged tail; the autotuner's
    choice is one of them."""
    inst = CASES[name]()
    kw = {"plain": {}, "smooth": {"alpha": 0.2}, "srmp": {"averaging": 1, "rank": "cm"}}[variant]
    a, b, c = solver(inst, staging=0, **kw), solver(inst, staging=1, **kw), solver(inst, staging=2, **kw)
    assert a.staging == 0 and b.staging == 1 | (1 << 2) and c.staging == 2 | (2 << 2)
    ta = _trace(a, 19)
    np.testing.assert_array_equal(ta, _trace(b, 19))
    np.testing.assert_array_equal(ta, _trace(c, 19))
    la, pa = a.get_state()
    for other in (b, c):
        lo, po = other.get_state()
        np.testing.assert_array_equal(la, lo)
        np.testing.assert_array_equal(pa, po)
    auto = solver(inst, **kw)
    assert (auto.staging & 3) <= 2 and (auto.staging >> 2) <= 2
    np.testing.assert_array_equal(_trace(auto, 19), _trace(solver(inst, staging=0, **kw), 19))


# ------------------------------------------------------------------------------------------
# lane tiles (one lane per BDD of width <= 2) against two-lane teams
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["potts_20x20x3", "matching_300x300", "matching_small", "tracking_10x40",
                                  "random_wide", "tomography_16"])
def test_lane_tiles_bit_identical_to_teams(lib, name):
    """BDDs whose layers have at most two nodes run one per lane (32 per warp) or as two-lane
    teams (16 per warp): the same operations in the same order, so bound traces, multipliers,
    pending sums and min-marginals are bit-identical, over 8-iteration graphs plus a ragged tail
    and for every staging variant of the other classes."""
    inst = CASES[name]()
    teams = solver(inst, lanes=0)
    assert teams.lanes == 0
    t_ref = _trace(teams, 19)
    l_ref, p_ref = teams.get_state()
    _, lam_ref, m0_ref, m1_ref = teams.iterate(0, lam=True, mm=True)
    for staging in (-1, 0, 1, 2):
        lanes = solver(inst, lanes=1, staging=staging)
        assert lanes.lanes == 1
        np.testing.assert_array_equal(_trace(lanes, 19), t_ref)
        la, pa = lanes.get_state()
        np.testing.assert_array_equal(la, l_ref)
        np.testing.assert_array_equal(pa, p_ref)
        _, lam_l, m0_l, m1_l = lanes.iterate(0, lam=True, mm=True)
        np.testing.assert_array_equal(lam_l, lam_ref)
        np.testing.assert_array_equal(m0_l, m0_ref)
        np.testing.assert_array_equal(m1_l, m1_ref)


def test_lane_tiles_default_and_refusals(lib):
    """Plain solvers without the layout tuner default to lane tiles (with it, lane tiles are one
    of its choices); smoothed, split, fused and persistent solvers keep the team layout, and
    asking them for lane tiles is refused."""
    from paper_2009_00481_gb300 import BDDError
    from paper_2009_00481_gb300.binding import BDD_EINVAL
    inst = CASES["potts_20x20x3"]()
    assert solver(inst, tune_layout=0).lanes == 1
    for kw in ({"alpha": 0.2}, {"split_depth": 2}, {"fused_pending": 1}, {"schedule": 0}):
        assert solver(inst, **kw).lanes == 0
        with pytest.raises(BDDError) as e:
            solver(inst, lanes=1, **kw)
        assert e.value.code == BDD_EINVAL


# ------------------------------------------------------------------------------------------
# the layout tuner: every table it may pick computes the same values
# ------------------------------------------------------------------------------------------

def _layout_tables():
    up, blk = [-1] * 28, [-1] * 28
    for k in range(28):
        c = k // 4
        if c <= 1:
            up[k], blk[k] = 7, 1
        elif c < 6:
            up[k], blk[k] = c + 1, 6
    return {"lanes_and_wider_teams": up, "teams_and_blocks": blk}


@pytest.mark.parametrize("name", ["potts_20x20x3", "matching_small", "tomography_16", "tracking_10x40",
                                  "random_wide"])
def test_layout_tuner_choices_bit_identical(lib, name):
    """The tuned layout and every alternative tile-class table (lane tiles or two-lane teams for
    widths <= 2, teams of 2^c or 2^(c+1) lanes, block tiles) give bit-identical bound traces,
    multipliers, pending sums and min-marginals; the tuned solver reports a class for every key
    that has nodes."""
    inst = CASES[name]()
    ref = solver(inst, tune_layout=0, lanes=0)
    t_ref = _trace(ref, 19)
    l_ref, p_ref = ref.get_state()
    _, _, m0_ref, m1_ref = ref.iterate(0, mm=True)
    tuned = solver(inst)
    rep = tuned.layout_table()
    assert np.all((rep["cls"] >= 0) == (rep["nodes"] > 0))
    others = [tuned] + [solver(inst, layout_classes=np.asarray(t, np.int32)) for t in _layout_tables().values()]
    for s in others:
        np.testing.assert_array_equal(_trace(s, 19), t_ref)
        la, pa = s.get_state()
        np.testing.assert_array_equal(la, l_ref)
        np.testing.assert_array_equal(pa, p_ref)
        _, _, m0, m1 = s.iterate(0, mm=True)
        np.testing.assert_array_equal(m0, m0_ref)
        np.testing.assert_array_equal(m1, m1_ref)
