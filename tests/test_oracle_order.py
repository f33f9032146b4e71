"""Pins for the variable order (Appendix A.3) and SRMP averaging (Appendix A.4) in the oracle."""
from __future__ import annotations

import numpy as np
import pytest

from instances import potts_mrf, random_ilp, tracking
from instances.generators import _from_rows
from oracle import ORC_EINVAL, Oracle, OracleError
from tests import bruteforce as bf


def _relabel(inst, perm):
    """The same ILP with variable i renamed perm[i]."""
    rows = [(perm[cols], vals, b, sense) for cols, vals, b, sense in inst.rows()]
    c = np.zeros(inst.n, np.float32)
    c[perm] = inst.c
    return _from_rows(inst.name + "_relabelled", inst.n, rows, c)


@pytest.mark.parametrize("srmp", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_schedules_match_enumeration(seed, srmp):
    """Alg. 1 and the deferred schedule under a random order, with eq. mma-update or
    eq. srmp-update, against the same schedules run with min-marginals from enumeration."""
    inst = random_ilp(n=11, m=8, max_row_vars=6, seed=40 + seed)
    rank = np.random.default_rng(seed).permutation(inst.n)
    o = Oracle(inst, rank=rank)
    if srmp:
        o.set_srmp()
    np.testing.assert_allclose(o.run_sequential(4), bf.sequential_enum(inst, 4, rank, srmp),
                               rtol=0, atol=1e-11)
    o.reset()
    np.testing.assert_allclose(o.run_parallel(6, omega=0.5),
                               bf.parallel_enum(inst, 6, 0.5, rank, srmp), rtol=0, atol=1e-11)


@pytest.mark.parametrize("srmp", [False, True])
def test_relabelling_is_exact(srmp):
    """Renaming variable i to perm[i] and ordering by the old index reproduces the identity-order
    run bit for bit (the bound up to the summation order over variables): the order alone
    decides layers and visits, never the names."""
    inst = potts_mrf(4, 4, 3, seed=3)
    perm = np.random.default_rng(1).permutation(inst.n)
    ren = _relabel(inst, perm)
    rank = np.empty(inst.n, np.int64)
    rank[perm] = np.arange(inst.n)
    a, b = Oracle(inst), Oracle(ren, rank=rank)
    if srmp:
        a.set_srmp()
        b.set_srmp()
    assert np.array_equal(a.run_sequential(5), b.run_sequential(5))
    a.reset()
    b.reset()
    ta, tb = a.run_parallel(12), b.run_parallel(12)
    assert np.array_equal(a.pending()[...], b.pending()[perm])  # every update bit for bit
    np.testing.assert_allclose(ta, tb, rtol=1e-14, atol=0)  # sum_i min(0, P_i) sums in index order


def test_order_does_not_change_the_subproblems():
    """Solution counts, energies and min-marginals of every row are properties of X_j and lambda
    alone (Sec. 3.2): any layer order gives the same values."""
    inst = random_ilp(n=20, m=10, max_row_vars=9, seed=77)
    lam = np.random.default_rng(3).normal(size=inst.nnz)
    base = Oracle(inst)
    base.set_state(lam)
    want = (base.counts(), base.energies(), *base.min_marginals(fold=False))
    for s in range(3):
        o = Oracle(inst, rank=np.random.default_rng(10 + s).permutation(inst.n))
        o.set_state(lam)
        got = (o.counts(), o.energies(), *o.min_marginals(fold=False))
        np.testing.assert_array_equal(got[0], want[0])
        for g, w in zip(got[1:], want[1:]):
            np.testing.assert_allclose(g, w, rtol=0, atol=1e-12)


def test_layers_follow_the_order():
    inst = tracking(frames=3, dets=5, seed=2)
    rank = np.random.default_rng(5).permutation(inst.n)
    can = Oracle(inst, rank=rank).canonical()
    o = 0
    for d in can["bdd_depth"]:
        v = can["occ_var"][o:o + d]
        assert np.all(np.diff(rank[v]) > 0)
        o += d
    ident = Oracle(inst, rank=np.arange(inst.n)).canonical()
    plain = Oracle(inst).canonical()
    for k in plain:
        assert np.array_equal(ident[k], plain[k])


@pytest.mark.parametrize("bad", [[0, 0, 1], [0, 1, 3], [-1, 0, 1]])
def test_rank_must_be_a_permutation(bad):
    inst = random_ilp(n=3, m=2, max_row_vars=3, seed=1)
    with pytest.raises(OracleError) as e:
        Oracle(inst, rank=np.array(bad))
    assert e.value.code == ORC_EINVAL


@pytest.mark.parametrize("seed", range(4))
def test_srmp_sequential_prop1(seed):
    """The SRMP update gains the same amount as eq. mma-update (Prop. 1): the subtracted
    differences equalise every min-marginal pair, and re-adding sum_k d_k on J_i^> alone
    changes the energy sum by min(0, sum_k d_k), whichever non-empty set receives it."""
    inst = random_ilp(n=18, m=12, max_row_vars=8, seed=600 + seed)
    o = Oracle(inst, rank=np.random.default_rng(seed).permutation(inst.n))
    o.set_srmp()
    tr = o.run_sequential(12, check=True)
    w = o.worst()
    assert w["prop1"] < 1e-10 and w["negative_gain"] < 1e-12
    assert w["monotone_drop"] < 1e-12 and w["invariant"] < 1e-12
    assert np.all(np.diff(tr) >= -1e-12 * np.maximum(1, np.abs(tr[1:])))


@pytest.mark.parametrize("seed", range(4))
def test_srmp_parallel_invariants(seed):
    inst = random_ilp(n=20, m=14, max_row_vars=9, seed=700 + seed)
    o = Oracle(inst)
    o.set_srmp()
    tr = o.run_parallel(20, omega=0.5, check=True)
    w = o.worst()
    assert w["incremental_mm"] < 1e-10 and w["invariant"] < 1e-12 and w["monotone_drop"] < 1e-12
    opt = bf.ilp_optimum(inst)
    assert tr.max() <= opt + 1e-9


def test_srmp_hand_example():
    """Rows A: x0 + x1 <= 1 and B: x0 <= 1, c = (-2, -1), one sequential iteration.  Start:
    lambda_A = (-1, -1), lambda_B0 = -1.  Forward at x0: d_A = 0, d_B = -1, S = -1; J_0^> = {A}
    (B has no later variable), so lambda_A0 = -2 and lambda_B0 = 0 (eq. mma-update would give
    -1.5 and -0.5).  Forward at x1: J_1^> is empty, fallback to J_1 = {A}: d = 1 = S, nothing
    moves.  Backward at x1: the same.  Backward at x0: J_0^< is empty, fallback to {A, B}:
    d_A = -1, d_B = 0, S = -1, so lambda_A0 = -1.5, lambda_B0 = -0.5; bound -2 = optimum."""
    inst = _from_rows("hand", 2, [(np.array([0, 1]), np.array([1, 1]), 1, -1),
                                  (np.array([0]), np.array([1]), 1, -1)],
                      np.array([-2.0, -1.0], np.float32))
    o = Oracle(inst)
    o.set_srmp()
    tr = o.run_sequential(1)
    np.testing.assert_allclose(o.lam(fold=False), [-1.5, -1.0, -0.5], rtol=0, atol=1e-15)
    assert abs(tr[0] - (-2.0)) < 1e-15
    # the forward half alone: the deferred schedule's first forward sweep takes no share
    # (P = 0), so the hand values of the forward pass are checked on the sequential schedule
    # through enumeration of the same instance
    D = bf.EnumDual(inst)
    assert D.weights(0, True, True) == [1.0, 0.0]
    assert D.weights(0, False, True) == [0.5, 0.5]
    assert D.weights(1, True, True) == [1.0]


def test_srmp_fold_keeps_the_invariant():
    """Folding the forward sweep's SRMP shares into lambda keeps sum_j lambda^j_i = c_i, puts
    nothing on a last-layer occurrence of a variable that has other occurrences in J_i^>, and
    equals the plain fold P_i / |J_i| when SRMP is off."""
    inst = tracking(frames=3, dets=6, seed=3)
    o = Oracle(inst)
    o.set_srmp()
    o.run_parallel(7, omega=0.5)
    lam, unf, P = o.lam(fold=True), o.lam(fold=False), o.pending()
    sums = np.zeros(inst.n)
    np.add.at(sums, inst.col, lam)
    deg = np.bincount(inst.col[inst.val != 0], minlength=inst.n)
    np.testing.assert_allclose(sums[deg > 0], inst.c[deg > 0], rtol=0, atol=1e-12)
    can = o.canonical()
    last = np.zeros(len(can["occ_var"]), bool)
    last[np.cumsum(can["bdd_depth"]) - 1] = True
    first = np.zeros_like(last)
    first[np.concatenate([[0], np.cumsum(can["bdd_depth"])[:-1]])] = True
    for occ in np.nonzero(last & ~first)[0]:
        i = can["occ_var"][occ]
        if np.any(~last[can["occ_var"] == i]):
            assert lam[can["occ_csr"][occ]] == unf[can["occ_csr"][occ]]
    p = Oracle(inst)
    p.set_state(unf, P)
    np.testing.assert_allclose(p.lam(fold=True), unf + (P / np.maximum(deg, 1))[inst.col], rtol=0, atol=1e-15)
