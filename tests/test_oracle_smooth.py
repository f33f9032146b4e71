"""Pins for the oracle's smoothed (log-sum-exp) algebra, Appendix A.5 and Table 3."""
from __future__ import annotations

import numpy as np
import pytest

from instances import potts_mrf, random_ilp, tracking
from oracle import Oracle
from tests import bruteforce as bf


def _lse_min(v, alpha):
    """-alpha log sum exp(-v / alpha) over a finite set, with the minimum factored out."""
    v = np.asarray(v, np.float64)
    if v.size == 0:
        return np.inf
    m = v.min()
    return m - alpha * np.log(np.exp(-(v - m) / alpha).sum())


@pytest.mark.parametrize("alpha", [0.05, 0.3, 2.0])
@pytest.mark.parametrize("seed", range(5))
def test_smoothed_energy_and_marginals_match_enumeration(seed, alpha):
    """eq. bdd-enery-smoothed and eq. marginal-log-sum-exp by enumeration of X_j."""
    inst = random_ilp(n=20, m=8, max_row_vars=10, seed=900 + seed)
    o = Oracle(inst)
    o.set_alpha(alpha)
    rng = np.random.default_rng(seed)
    lam = rng.normal(size=inst.nnz)
    o.set_state(lam)
    E = o.energies()
    m0, m1 = o.min_marginals(fold=False)
    for j, (cols, vals, b, sense) in enumerate(inst.rows()):
        order = np.argsort(cols, kind="stable")
        pos = inst.row_ptr[j] + order
        X = bf.assignments(len(cols))
        feas = bf.row_feasible(vals[order], b, sense)
        cost = X @ lam[pos]
        assert abs(E[j] - _lse_min(cost[feas], alpha)) < 1e-10
        for t in range(len(cols)):
            for beta, got in ((0, m0), (1, m1)):
                want = _lse_min(cost[feas & (X[:, t] == beta)], alpha)
                if np.isinf(want):
                    assert np.isinf(got[pos[t]])
                else:
                    assert abs(got[pos[t]] - want) < 1e-10


@pytest.mark.parametrize("alpha", [0.01, 0.1, 1.0])
def test_prop5_sandwich(alpha):
    """Prop. 5: E^j >= E^j_alpha >= E^j - alpha log |X_j| for every BDD (the paper's strict
    first inequality needs |X_j| >= 2: a single feasible point gives equality)."""
    inst = random_ilp(n=24, m=12, max_row_vars=12, seed=17)
    rng = np.random.default_rng(2)
    lam = rng.normal(size=inst.nnz)
    o = Oracle(inst)
    o.set_state(lam)
    E = o.energies()
    cnt = o.counts()
    o.set_alpha(alpha)
    o.set_state(lam)
    Ea = o.energies()
    assert np.all(E >= Ea - 1e-12)
    assert np.all(Ea >= E - alpha * np.log(cnt) - 1e-12)
    if alpha >= 0.1:
        assert np.all((E > Ea)[cnt >= 2])
    assert np.all(np.abs(E - Ea)[cnt == 1] < 1e-12)


def test_alpha_to_zero_recovers_min_sum():
    """As alpha -> 0 the smoothed schedule becomes the min-sum schedule."""
    inst = potts_mrf(5, 5, 3, seed=4)
    plain = Oracle(inst).run_parallel(30, omega=0.5)
    o = Oracle(inst)
    o.set_alpha(1e-7)
    soft = o.run_parallel(30, omega=0.5)
    np.testing.assert_allclose(soft, plain, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("alpha", [0.05, 0.5])
def test_smoothed_schedule_invariants(alpha):
    """Smoothed deferred schedule: incremental marginals equal the definitional smoothed
    marginals at every visit, sum_j lambda + P = c, and the smoothed bound is below the plain
    bound of the same state."""
    inst = tracking(frames=3, dets=6, seed=3)
    o = Oracle(inst)
    o.set_alpha(alpha)
    tr = o.run_parallel(15, omega=0.5, check=True)
    w = o.worst()
    assert w["incremental_mm"] < 1e-10 and w["invariant"] < 1e-12
    lam, P = o.lam(fold=False), o.pending()
    p = Oracle(inst)
    p.set_state(lam, P)
    assert tr[-1] <= p.bound() + 1e-12
