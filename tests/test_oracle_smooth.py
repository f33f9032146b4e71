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


# ------------------------------------------------------------------------------------------
# FP64 gradient of the smoothed bound (reverse mode through the deferred schedule)
# ------------------------------------------------------------------------------------------

def _smoothed_bound(inst, c, alpha, K, srmp=False, lib=None):
    import copy
    j = copy.copy(inst)
    j.c = np.asarray(c, np.float64)
    o = Oracle(j, lib=lib)
    if srmp:
        o.set_srmp(True)
    o.set_alpha(alpha)
    return float(o.run_parallel(K, omega=0.5)[-1]) if K > 0 else o.bound()


def _central_differences(inst, alpha, K, srmp=False, h=1e-6, lib=None):
    c0 = inst.c.astype(np.float64)
    fd = np.zeros(inst.n)
    for i in range(inst.n):
        cp, cm = c0.copy(), c0.copy()
        cp[i] += h
        cm[i] -= h
        fd[i] = (_smoothed_bound(inst, cp, alpha, K, srmp, lib) - _smoothed_bound(inst, cm, alpha, K, srmp, lib)) / (2 * h)
    return fd


def _oracle_gradient(inst, alpha, K, srmp=False, lib=None):
    o = Oracle(inst, lib=lib)
    if srmp:
        o.set_srmp(True)
    o.set_alpha(alpha)
    return o.smooth_gradient(K, omega=0.5)


GRAD_CASES = {
    "tracking_3x6": lambda: tracking(frames=3, dets=6, seed=0),
    "potts_3x3x3": lambda: potts_mrf(3, 3, 3, seed=1),
    "random_ilp": lambda: random_ilp(n=20, m=8, max_row_vars=10, seed=3),
}


@pytest.mark.parametrize("srmp", [False, True])
@pytest.mark.parametrize("K", [1, 6])
@pytest.mark.parametrize("alpha", [0.1, 0.5])
@pytest.mark.parametrize("name", sorted(GRAD_CASES))
def test_oracle_gradient_matches_central_differences(name, alpha, K, srmp):
    """Every coordinate of the reverse-mode gradient against FP64 central differences of the
    oracle's own smoothed bound (h = 1e-6: truncation and rounding error both below 1e-8 here);
    the bound it returns is the last entry of the schedule's trace, bit for bit."""
    inst = GRAD_CASES[name]()
    lb, g = _oracle_gradient(inst, alpha, K, srmp)
    assert lb == _smoothed_bound(inst, inst.c, alpha, K, srmp)
    fd = _central_differences(inst, alpha, K, srmp)
    scale = max(1.0, np.abs(fd).max())
    err = np.abs(g - fd).max() / scale
    assert err < 1e-6, err


@pytest.mark.parametrize("alpha", [0.05, 0.3, 2.0])
def test_oracle_gradient_at_zero_iterations_is_gibbs_marginals(alpha):
    """K = 0: the bound is sum_j E_alpha^j(c/|J|) plus the soft slack terms, and d/dc_i is the
    average over j in J_i of the Gibbs probability Pr_j(x_i = 1) under exp(-lambda^j x / alpha)
    on X_j (the derivative of -alpha log sum exp), by enumeration; a variable in no row gets
    the derivative of the soft minimum of {0, c_i}, 1 / (1 + exp(c_i / alpha))."""
    from instances.generators import _from_rows
    base = random_ilp(n=14, m=6, max_row_vars=9, seed=21, coef=3)
    rows = list(base.rows())
    c = np.concatenate([base.c, np.array([0.7, -1.3], np.float32)])  # two variables in no row
    inst = _from_rows("gibbs", base.n + 2, rows, c)
    lb, g = _oracle_gradient(inst, alpha, 0)
    deg = np.zeros(inst.n)
    for cols, vals, b, sense in rows:
        deg[cols[vals != 0]] += 1
    want = np.zeros(inst.n)
    bound = 0.0
    for cols, vals, b, sense in rows:
        keep = vals != 0
        cols, vals = cols[keep], vals[keep]
        X = bf.assignments(len(cols))
        feas = bf.row_feasible(vals, b, sense)
        lam = inst.c[cols].astype(np.float64) / deg[cols]
        cost = X[feas] @ lam
        m = cost.min()
        w = np.exp(-(cost - m) / alpha)
        bound += m - alpha * np.log(w.sum())
        want[cols] += (w @ X[feas]) / w.sum() / deg[cols]
    for i in np.nonzero(deg == 0)[0]:
        ci = float(inst.c[i])
        want[i] = 1.0 / (1.0 + np.exp(ci / alpha))
        bound += min(0.0, ci) - alpha * np.log1p(np.exp(-abs(ci) / alpha))
    bound += (deg > 0).sum() * (-alpha * np.log(2.0))  # soft minimum of {0, P_i = 0}
    assert abs(lb - bound) < 1e-10 * max(1.0, abs(bound))
    np.testing.assert_allclose(g, want, rtol=0, atol=1e-12)
