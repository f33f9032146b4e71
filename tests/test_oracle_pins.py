"""Pins for the FP64 oracle: each test checks the oracle against something other than itself
(the paper's worked example, enumeration, closed forms, duality, LP, invariants)."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

from instances import (SENSE_EQ, SENSE_GE, SENSE_LE, Instance, potts_mrf, random_ilp,
                       sparse_matching, tomography)
from instances.generators import _from_rows
from oracle import ORC_EINFEASIBLE, ORC_EINVAL, Oracle, OracleError
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def single_row(cols, vals, b, sense, n=None, c=None):
    n = n if n is not None else (max(cols) + 1 if len(cols) else 1)
    c = np.zeros(n, np.float32) if c is None else c
    return _from_rows("row", n, [(np.asarray(cols), np.asarray(vals), b, sense)], c)


# ------------------------------------------------------------------------------------------
# BDD construction
# ------------------------------------------------------------------------------------------

def test_fig1_worked_example():
    """Sec. 5.1 Figure 1: x1 + x3 + x7 = 1 gives exactly the drawn five-node BDD."""
    g = json.load(open(os.path.join(GOLDEN, "fig1_bdd.json")))
    r = g["row"]
    o = Oracle(single_row(r["cols"], r["vals"], r["b"], r["sense"], n=r["n"]))
    canon = o.canonical()
    assert o.N == 5 and o.nb == 1
    layers = bf.split_bdds(canon)[0]
    assert len(layers) == len(g["layers"])
    for got, want in zip(layers, g["layers"]):
        assert got["var"] == want["var"]
        assert got["lo"].tolist() == want["lo"]
        assert got["hi"].tolist() == want["hi"]
        assert got["minsum"].tolist() == want["minsum"]
    ok, _ = bf.walk(layers, g["marked_path"]["x"])
    assert ok == g["marked_path"]["accepted"]


@pytest.mark.parametrize("seed", range(40))
def test_bdd_matches_enumeration(seed):
    """Def. 4 and Prop. 2: the BDD accepts exactly the feasible set; every layer has as many
    nodes as there are distinct non-false subfunctions (reduced, non-skipping); nodes are in
    ascending smallest-partial-sum order and that sum is the true minimum over prefixes."""
    rng = np.random.default_rng(1000 + seed)
    k = int(rng.integers(1, 13))
    vals = rng.integers(1, 4, size=k) * rng.choice([-1, 1], size=k)
    sense = int(rng.choice([SENSE_LE, SENSE_EQ, SENSE_GE]))
    x0 = rng.integers(0, 2, size=k)
    b = int(vals @ x0) + (int(rng.integers(-2, 3)) if sense != SENSE_EQ else 0)
    cols = np.sort(rng.choice(40, size=k, replace=False))
    feas = bf.row_feasible(vals, b, sense)
    try:
        o = Oracle(single_row(cols, vals, b, sense, n=40))
    except OracleError as e:
        assert e.code == ORC_EINFEASIBLE and not feas.any()
        return
    layers = bf.split_bdds(o.canonical())[0]
    assert [lay["var"] for lay in layers] == cols.tolist()
    X = bf.assignments(k)
    acc = np.array([bf.walk(layers, x)[0] for x in X])
    assert np.array_equal(acc, feas)
    for l in range(k):
        assert len(layers[l]["lo"]) == bf.layer_subfunction_count(feas, k, l), l
    # canonical order: smallest partial sum per node, strictly ascending inside a layer
    minsum = [dict() for _ in range(k)]
    for x in X:
        _, path = bf.walk(layers, x)
        s = 0
        for l, node in enumerate(path):
            minsum[l][node] = min(minsum[l].get(node, s), s)
            s += int(vals[l]) * int(x[l])
    for l in range(k):
        want = [minsum[l][v] for v in range(len(layers[l]["lo"]))]
        assert layers[l]["minsum"].tolist() == want
        assert all(a < b_ for a, b_ in zip(want, want[1:]))


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 13])
def test_closed_form_node_counts(k):
    """sum of k variables = 1 and <= 1 both have 2k-1 nodes (Figure 1 is k = 3);
    sum_{l} y_l - x = 0 with x first has 2k+1 nodes."""
    cols = list(range(k))
    assert Oracle(single_row(cols, [1] * k, 1, SENSE_EQ)).N == 2 * k - 1
    assert Oracle(single_row(cols, [1] * k, 1, SENSE_LE)).N == 2 * k - 1
    cols = list(range(k + 1))
    assert Oracle(single_row(cols, [-1] + [1] * k, 0, SENSE_EQ)).N == 2 * k + 1


def test_potts_config_node_count():
    """The 20x20x3 Potts MRF: 400 one-hot rows of 5 nodes and 4560 marginalisation rows of
    7 nodes = 33,920 nodes."""
    o = Oracle(potts_mrf(20, 20, 3, seed=0))
    assert (o.nb, o.O, o.N) == (4960, 19440, 33920)


def test_input_errors():
    # duplicate (j, i)
    with pytest.raises(OracleError) as e:
        Oracle(single_row([1, 1], [1, 1], 1, SENSE_LE, n=3))
    assert e.value.code == ORC_EINVAL
    # infeasible row reports its id
    inst = _from_rows("inf", 3, [(np.array([0, 1]), np.array([1, 1]), 1, SENSE_LE),
                                 (np.array([0, 2]), np.array([1, 1]), 3, SENSE_EQ)],
                      np.zeros(3, np.float32))
    with pytest.raises(OracleError) as e:
        Oracle(inst)
    assert e.value.code == ORC_EINFEASIBLE and e.value.row == 1
    # non-finite cost
    with pytest.raises(OracleError) as e:
        Oracle(single_row([0], [1], 1, SENSE_LE, c=np.array([np.nan], np.float32)))
    assert e.value.code == ORC_EINVAL
    # empty rows: dropped when 0 (sense) b holds, infeasible otherwise
    ok = _from_rows("e", 2, [(np.array([], np.int64), np.array([], np.int64), 0, SENSE_LE),
                             (np.array([0, 1]), np.array([0, 1]), 1, SENSE_EQ)],
                    np.zeros(2, np.float32))
    o = Oracle(ok)
    assert o.nb == 1 and o.O == 1  # the zero coefficient is not an occurrence
    bad = _from_rows("e", 1, [(np.array([], np.int64), np.array([], np.int64), 1, SENSE_EQ)],
                     np.zeros(1, np.float32))
    with pytest.raises(OracleError) as e:
        Oracle(bad)
    assert e.value.code == ORC_EINFEASIBLE


# ------------------------------------------------------------------------------------------
# Min-marginals, energies and counts
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_min_marginals_match_enumeration(seed):
    """eqs. arc-marginal / marginal-aggregation (Sec. 5.3) give the min-marginals of
    eq. min-marginals (Sec. 3.2); E^j is the minimum over X_j; counts are |X_j| (Table 3)."""
    inst = random_ilp(n=24, m=10, max_row_vars=12, seed=seed)
    o = Oracle(inst)
    rng = np.random.default_rng(seed)
    lam = rng.normal(size=inst.nnz)
    o.set_state(lam)
    m0, m1 = o.min_marginals(fold=False)
    E = o.energies()
    cnt = o.counts()
    for j, (cols, vals, b, sense) in enumerate(inst.rows()):
        order = np.argsort(cols, kind="stable")
        pos = inst.row_ptr[j] + order
        em0, em1, eE, ecnt = bf.min_marginals_enum(vals[order], b, sense, lam[pos])
        np.testing.assert_allclose(m0[pos], em0, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(m1[pos], em1, rtol=1e-12, atol=1e-12)
        assert abs(E[j] - eE) < 1e-12
        assert cnt[j] == ecnt


def test_forced_variable_has_infinite_min_marginal():
    """x0 + x1 = 2 forces both variables to 1: the 0-min-marginal is +inf."""
    o = Oracle(single_row([0, 1], [1, 1], 2, SENSE_EQ, c=np.array([1.0, -2.0], np.float32)))
    m0, m1 = o.min_marginals(fold=False)
    assert np.isinf(m0).all() and np.allclose(m1, [-1.0, -1.0])


# ------------------------------------------------------------------------------------------
# Schedules: Alg. 1 (sequential) and the parallel deferred-averaging schedule
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_sequential_prop1_and_monotone(seed):
    """Alg. 1: every update gains exactly the Prop. 1 amount (when all min-marginals are
    finite) and never loses; the bound never decreases; sum_j lambda^j_i = c_i."""
    inst = random_ilp(n=18, m=12, max_row_vars=8, seed=100 + seed)
    o = Oracle(inst)
    tr = o.run_sequential(15, check=True)
    w = o.worst()
    assert w["prop1"] < 1e-10 and w["negative_gain"] < 1e-12
    assert w["monotone_drop"] < 1e-12 and w["invariant"] < 1e-12
    assert np.all(np.diff(tr) >= -1e-12 * np.maximum(1, np.abs(tr[1:])))


@pytest.mark.parametrize("omega", [0.5, 1.0])
@pytest.mark.parametrize("seed", range(6))
def test_parallel_schedule_invariants(seed, omega):
    """Deferred-averaging schedule: incremental min-marginals (Prop. 3) equal the definitional
    ones at every visit, sum_j lambda^j_i + P_i = c_i after every sweep, and the y-slack bound
    (Appendix A.1) never decreases."""
    inst = random_ilp(n=20, m=14, max_row_vars=9, seed=200 + seed)
    o = Oracle(inst)
    tr = o.run_parallel(20, omega=omega, check=True)
    w = o.worst()
    assert w["incremental_mm"] < 1e-10
    assert w["invariant"] < 1e-12
    assert w["monotone_drop"] < 1e-12
    assert np.all(np.diff(tr) >= -1e-12 * np.maximum(1, np.abs(tr[1:])))


def test_parallel_schedule_hand_example():
    """Two rows x0 <= 1 share x0 with c0 = -1: lambda = (-0.5, -0.5), each BDD has m0 = 0,
    m1 = -0.5.  With omega = 0.5 one forward sweep moves each lambda to -0.25 and P to -0.5,
    so the bound is E_A + E_B + min(0, P) = -0.25 - 0.25 - 0.5 = -1 = the optimum."""
    inst = _from_rows("hand", 1, [(np.array([0]), np.array([1]), 1, SENSE_LE),
                                  (np.array([0]), np.array([1]), 1, SENSE_LE)],
                      np.array([-1.0], np.float32))
    o = Oracle(inst)
    assert abs(o.bound() - (-1.0)) < 1e-15  # E = -0.5 each at the start
    tr = o.run_parallel(3, omega=0.5)
    assert np.allclose(tr, -1.0)
    np.testing.assert_allclose(o.lam(fold=False), [-0.25, -0.25])
    np.testing.assert_allclose(o.pending(), [-0.5])
    np.testing.assert_allclose(o.lam(fold=True), [-0.5, -0.5])


@pytest.mark.parametrize("seed", range(10))
def test_weak_duality_bruteforce(seed):
    """Any dual bound is <= the ILP optimum (Sec. 3.1): brute force over {0,1}^n."""
    inst = random_ilp(n=16, m=10, max_row_vars=7, seed=300 + seed)
    opt = bf.ilp_optimum(inst)
    o = Oracle(inst)
    trp = o.run_parallel(30, omega=0.5)
    o.reset()
    trs = o.run_sequential(10)
    assert trp.max() <= opt + 1e-9
    assert trs.max() <= opt + 1e-9


@pytest.mark.parametrize("H,W,seed", [(2, 2, 0), (2, 3, 1), (3, 3, 2)])
def test_potts_bound_below_map(H, W, seed):
    """Potts MRF (Appendix E.1 formulation): the bound stays below the minimum labeling energy."""
    inst = potts_mrf(H, W, 2, seed=seed)
    opt = bf.potts_map(H, W, 2, inst.c)
    o = Oracle(inst)
    tr = o.run_parallel(200, omega=0.5)
    assert tr.max() <= opt + 1e-9
    o.reset()
    trs = o.run_sequential(50)
    assert trs.max() <= opt + 1e-9


def test_chain_mrf_reaches_map():
    """A 1x6 chain with 3 labels: the local polytope is tight on trees, so the bound stays
    below the MAP energy and (for this seed) closes the gap to within 1e-6."""
    inst = potts_mrf(1, 6, 3, seed=5)
    opt = bf.potts_map(1, 6, 3, inst.c)
    o = Oracle(inst)
    tr = o.run_sequential(200)
    assert tr.max() <= opt + 1e-9
    assert opt - tr[-1] < 1e-6


def _lp_optimum(inst):
    from scipy.optimize import linprog
    from scipy.sparse import csr_matrix
    A = csr_matrix((inst.val.astype(np.float64), inst.col, inst.row_ptr), shape=(inst.m, inst.n))
    le, eq, ge = inst.sense == SENSE_LE, inst.sense == SENSE_EQ, inst.sense == SENSE_GE
    from scipy.sparse import vstack
    A_ub = vstack([A[le], -A[ge]])
    b_ub = np.concatenate([inst.b[le], -inst.b[ge]]).astype(np.float64)
    res = linprog(inst.c.astype(np.float64), A_ub=A_ub if A_ub.shape[0] else None,
                  b_ub=b_ub if A_ub.shape[0] else None, A_eq=A[eq], b_eq=inst.b[eq].astype(np.float64),
                  bounds=(0, 1), method="highs")
    assert res.status == 0
    return float(res.fun)


@pytest.mark.parametrize("which", ["potts", "matching"])
def test_bound_below_lp(which):
    """Rows with coefficients in {0, +-1} are totally unimodular one at a time, so the dual (D)
    optimum equals the LP relaxation optimum; every iterate is below it (HiGHS LP)."""
    if which == "potts":
        inst = potts_mrf(8, 8, 3, seed=3)
    else:
        inst = sparse_matching(n_left=40, n_right=40, k=5, n_pairs=300, seed=4)
    lp = _lp_optimum(inst)
    o = Oracle(inst)
    tr = o.run_parallel(300, omega=0.5)
    assert tr.max() <= lp + 1e-7 * max(1, abs(lp))
    # the method makes real progress towards the LP value (gap reported in the message)
    gap0 = lp - tr[0]
    gap = lp - tr[-1]
    assert gap < 0.5 * gap0, (gap0, gap)


def test_tomography_short_diagonals_force_variables():
    """A corner diagonal of length 1 with projection value 2 forces its pixel to level 2:
    the BDD of that row has a single path and the 0-min-marginal of x[pixel,2] is +inf."""
    inst = tomography(side=8, seed=0)
    o = Oracle(inst)
    m0, m1 = o.min_marginals(fold=False)
    gt = inst.meta["ground_truth"]
    # anti-diagonal / diagonal rows of length 1 exist at the corners
    assert np.isinf(m0).any() or np.isinf(m1).any() or gt.size == 0
    tr = o.run_parallel(20, omega=0.5, check=True)
    w = o.worst()
    assert w["monotone_drop"] < 1e-12 and w["invariant"] < 1e-12 and w["incremental_mm"] < 1e-10


def test_openmp_build_is_bit_identical():
    """The oracle's OpenMP build (the benchmark's second CPU baseline) runs schedule P's loops
    over BDDs and variables on all host cores and gives the single-threaded build's results bit
    for bit (traces, multipliers, pending sums), with and without SRMP."""
    import numpy as np

    from instances import config, tracking
    from oracle import Oracle, load_omp
    for inst in (config(0), tracking(frames=6, dets=30, seed=4)):
        for srmp in (False, True):
            a, b = Oracle(inst), Oracle(inst, lib=load_omp())
            if srmp:
                a.set_srmp(True)
                b.set_srmp(True)
            np.testing.assert_array_equal(a.run_parallel(25, omega=0.5), b.run_parallel(25, omega=0.5))
            np.testing.assert_array_equal(a.lam(fold=False), b.lam(fold=False))
            np.testing.assert_array_equal(a.pending(), b.pending())
