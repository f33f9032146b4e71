"""Pins for the oracle's sub-BDDs and copy-arc duals (Sec. 6: sub-BDDs, copy-arcs, the parallel
averaging algorithm, Prop. 4)."""
from __future__ import annotations

import numpy as np
import pytest

from instances import SENSE_EQ, SENSE_GE, SENSE_LE, potts_mrf, random_ilp, tomography
from instances.generators import _from_rows
from oracle import Oracle
from tests import bruteforce as bf


def _pairs_of_cut(layers, l_cut):
    """Copy pairs of the cut before layer l_cut, in the oracle's order (tails in node order,
    0-arc before 1-arc): list of (tail, side)."""
    out = []
    lay = layers[l_cut - 1]
    for u in range(len(lay["lo"])):
        for side, arr in ((0, lay["lo"]), (1, lay["hi"])):
            if arr[u] >= 0:
                out.append((u, side))
    return out


def _piece_energies_enum(vals, b, sense, lam, cuts_layers, mu_bar, mu, layers):
    """Energy of every piece of one row by enumeration: min over feasible x of (mu of the entry
    pair x uses + sum of lam x over the piece's layers + mu_bar of the exit pair)."""
    k = len(vals)
    X = bf.assignments(k)
    feas = bf.row_feasible(vals, b, sense)
    bounds = [0] + list(cuts_layers) + [k]
    pair_index = []  # per cut: dict (tail, side) -> global pair index
    base = 0
    for lc in cuts_layers:
        prs = _pairs_of_cut(layers, lc)
        pair_index.append({p: base + t for t, p in enumerate(prs)})
        base += len(prs)
    E = np.full(len(bounds) - 1, np.inf)
    for x, ok in zip(X, feas):
        if not ok:
            continue
        acc, path = bf.walk(layers, x)
        assert acc
        used = [pair_index[c][(path[lc - 1], int(x[lc - 1]))] for c, lc in enumerate(cuts_layers)]
        for p in range(len(bounds) - 1):
            cost = float(np.dot(lam[bounds[p]:bounds[p + 1]], x[bounds[p]:bounds[p + 1]]))
            if p > 0:
                cost += mu[used[p - 1]]
            if p < len(bounds) - 2:
                cost += mu_bar[used[p]]
            E[p] = min(E[p], cost)
    return E


@pytest.mark.parametrize("seed", range(12))
def test_piece_energies_match_enumeration(seed):
    """One row split at one or two random places; random lambda and random copy duals: every
    piece's energy (multi-root pieces with root messages min mu, copy arcs into top with cost
    mu_bar) equals the enumeration of the row's feasible points."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(4, 11))
    vals = rng.integers(1, 4, size=k) * rng.choice([-1, 1], size=k)
    sense = [SENSE_LE, SENSE_EQ, SENSE_GE][seed % 3]
    b = int(vals @ rng.integers(0, 2, size=k))
    inst = _from_rows("r", k, [(np.arange(k), vals, b, sense)], np.zeros(k, np.float32))
    layers = bf.split_bdds(Oracle(inst).canonical())[0]
    ncut = 1 + seed % 2
    cuts_layers = sorted(rng.choice(np.arange(1, k), size=ncut, replace=False).tolist())
    o = Oracle(inst)
    assert o.split(cuts_layers) == ncut + 1
    lam = rng.normal(size=k)
    o.set_state(lam)
    mb = rng.normal(size=o.npairs)
    mu = rng.normal(size=o.npairs)
    o.set_copy_duals(mb, mu)
    want = _piece_energies_enum(vals, b, sense, lam, cuts_layers, mb, mu, layers)
    np.testing.assert_allclose(o.energies(), want, rtol=0, atol=1e-12)


def test_no_cuts_is_the_unsplit_method():
    inst = random_ilp(n=16, m=10, max_row_vars=8, seed=5)
    a, b = Oracle(inst), Oracle(inst)
    assert b.split([]) == a.nb
    assert np.array_equal(a.run_parallel(25), b.run_parallel(25))


@pytest.mark.parametrize("gamma", [0.5, 1.0])
@pytest.mark.parametrize("seed", range(6))
def test_split_schedule_invariants_and_duality(seed, gamma):
    """With cuts: incremental min-marginals equal the definitional ones of the pieces at every
    visit, sum_j lambda + P = c, the bound never decreases (Prop. 4 together with the deferred
    averaging), mu + mu_bar <= 0 for every pair, and every bound is below the ILP optimum."""
    inst = random_ilp(n=15, m=10, max_row_vars=9, seed=40 + seed)
    rng = np.random.default_rng(seed)
    cuts = sorted(rng.choice(np.arange(1, inst.n), size=2, replace=False).tolist())
    o = Oracle(inst)
    o.split(cuts, gamma)
    tr = o.run_parallel(40, omega=0.5, check=True)
    w = o.worst()
    assert w["incremental_mm"] < 1e-10 and w["invariant"] < 1e-12 and w["monotone_drop"] < 1e-12
    mb, mu = o.copy_duals()
    assert np.all(mb + mu <= 1e-12)
    assert tr.max() <= bf.ilp_optimum(inst) + 1e-9


def test_split_bound_below_unsplit_at_start_and_converges():
    """The pieces relax the rows (copy constraints dualised): at mu = 0 the split bound is at most
    the unsplit one; iterating closes most of the gap."""
    inst = tomography(side=12, seed=3, unary_sigma=0.1)
    a = Oracle(inst)
    b = Oracle(inst)
    b.split([inst.n // 4, inst.n // 2, 3 * inst.n // 4])
    assert b.bound() <= a.bound() + 1e-9
    ta, tb = a.run_parallel(300), b.run_parallel(300)
    assert tb[-1] > tb[0] and (ta[-1] - tb[-1]) < 0.2 * (ta[-1] - tb[0])


def test_split_rejects_bad_input():
    inst = potts_mrf(3, 3, 2, seed=0)
    for cuts, g in (([0], 0.5), ([3, 3], 0.5), ([inst.n], 0.5), ([2], 0.0), ([2], 1.5)):
        with pytest.raises(ValueError):
            Oracle(inst).split(cuts, g)


def _pieces_by_row(can):
    """Depths of the pieces of every row, in layer order."""
    out = {}
    for r, d in zip(can["bdd_row"], can["bdd_depth"]):
        out.setdefault(int(r), []).append(int(d))
    return out


@pytest.mark.parametrize("D", [1, 2, 3, 5, 8])
def test_depth_split_structure(D):
    """Every piece has at most D layers, a row of k layers has ceil(k / D) pieces whose depths
    differ by at most one and add up to k, and the pieces keep the row's nodes and arcs: every
    copy code replaces one arc into a node of the next layer, in pair order."""
    inst = random_ilp(n=24, m=14, max_row_vars=12, seed=90 + D, coef=3)
    whole = Oracle(inst).canonical()
    o = Oracle(inst)
    o.split_depth(D)
    can = o.canonical()
    assert can["bdd_depth"].max() <= D
    k_of_row = dict(zip(whole["bdd_row"].tolist(), whole["bdd_depth"].tolist()))
    for r, ds in _pieces_by_row(can).items():
        k = k_of_row[r]
        assert sum(ds) == k and len(ds) == -(-k // D) and max(ds) - min(ds) <= 1, (r, k, ds)
    np.testing.assert_array_equal(can["occ_width"], whole["occ_width"])
    for side in ("lo", "hi"):
        c = can[side] <= -4
        assert np.all(whole[side][c] >= 0), "a copy arc replaced an arc into a terminal"
        np.testing.assert_array_equal(can[side][~c], whole[side][~c])
    codes = np.sort(np.concatenate([can["lo"][can["lo"] <= -4], can["hi"][can["hi"] <= -4]]))[::-1]
    np.testing.assert_array_equal(-4 - codes, np.arange(o.npairs))


@pytest.mark.parametrize("seed", range(8))
def test_depth_split_piece_energies_match_enumeration(seed):
    """One row cut into pieces of at most D layers; random lambda and copy duals: every piece's
    energy equals the enumeration of the row's feasible points (cut layers read from the
    pieces' depths)."""
    rng = np.random.default_rng(100 + seed)
    k = int(rng.integers(5, 12))
    vals = rng.integers(1, 4, size=k) * rng.choice([-1, 1], size=k)
    sense = [SENSE_LE, SENSE_EQ, SENSE_GE][seed % 3]
    b = int(vals @ rng.integers(0, 2, size=k))
    inst = _from_rows("r", k, [(np.arange(k), vals, b, sense)], np.zeros(k, np.float32))
    layers = bf.split_bdds(Oracle(inst).canonical())[0]
    D = int(rng.integers(2, k))
    o = Oracle(inst)
    o.split_depth(D)
    depths = o.canonical()["bdd_depth"]
    cuts_layers = np.cumsum(depths)[:-1].tolist()
    assert len(cuts_layers) >= 1
    lam = rng.normal(size=k)
    o.set_state(lam)
    mb = rng.normal(size=o.npairs)
    mu = rng.normal(size=o.npairs)
    o.set_copy_duals(mb, mu)
    want = _piece_energies_enum(vals, b, sense, lam, cuts_layers, mb, mu, layers)
    np.testing.assert_allclose(o.energies(), want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("D", [2, 4])
@pytest.mark.parametrize("seed", range(4))
def test_depth_split_schedule_invariants_and_duality(seed, D):
    """Depth split: incremental min-marginals equal the definitional ones at every visit, the
    invariant, a non-decreasing bound (Prop. 4's argument per cut), mu + mu_bar <= 0, weak
    duality; a depth limit no BDD exceeds changes nothing."""
    inst = random_ilp(n=15, m=10, max_row_vars=9, seed=60 + seed)
    o = Oracle(inst)
    o.split_depth(D)
    assert o.npairs > 0
    tr = o.run_parallel(40, omega=0.5, check=True)
    w = o.worst()
    assert w["incremental_mm"] < 1e-10 and w["invariant"] < 1e-12 and w["monotone_drop"] < 1e-12
    mb, mu = o.copy_duals()
    assert np.all(mb + mu <= 1e-12)
    assert tr.max() <= bf.ilp_optimum(inst) + 1e-9
    a, b = Oracle(inst), Oracle(inst)
    assert b.split_depth(100) == a.nb and b.npairs == 0
    assert np.array_equal(a.run_parallel(20), b.run_parallel(20))


def test_depth_split_closes_the_gap_on_tomography():
    """Tomography projections (up to 24 layers at side 12) in pieces of at most 6 layers: the
    bound starts no higher than the unsplit one and iterating closes most of the gap."""
    inst = tomography(side=12, seed=3, unary_sigma=0.1)
    a, b = Oracle(inst), Oracle(inst)
    b.split_depth(6)
    assert b.canonical()["bdd_depth"].max() <= 6
    assert b.bound() <= a.bound() + 1e-9
    ta, tb = a.run_parallel(300), b.run_parallel(300)
    assert tb[-1] > tb[0] and (ta[-1] - tb[-1]) < 0.2 * (ta[-1] - tb[0])


def test_depth_split_rejects_bad_input():
    inst = potts_mrf(3, 3, 2, seed=0)
    for D, g in ((0, 0.5), (-1, 0.5), (2, 0.0), (2, 1.5)):
        with pytest.raises(ValueError):
            Oracle(inst).split_depth(D, g)


@pytest.mark.parametrize("seed", range(3))
def test_split_with_srmp_keeps_the_checks(seed):
    """SRMP averaging (Appendix A.4) on pieces: a piece's first and last layers define its J_i^<
    and J_i^> membership.  Incremental min-marginals equal the definitional ones, the invariant
    and monotonicity hold, and the bound stays below the ILP optimum."""
    inst = random_ilp(n=15, m=10, max_row_vars=9, seed=80 + seed)
    o = Oracle(inst)
    o.set_srmp(True)
    o.split_depth(3)
    tr = o.run_parallel(30, omega=0.5, check=True)
    w = o.worst()
    assert w["incremental_mm"] < 1e-10 and w["invariant"] < 1e-12 and w["monotone_drop"] < 1e-12
    assert tr.max() <= bf.ilp_optimum(inst) + 1e-9


def test_copy_dual_sums_after_each_step():
    """From zero duals, after the forward copy step every pair's mu + mu_bar is -gamma times a
    nonnegative difference (so it never turns positive), and after the backward step too."""
    inst = random_ilp(n=14, m=9, max_row_vars=9, seed=91)
    o = Oracle(inst)
    o.split_depth(3, 0.5)
    for _ in range(15):
        o.run_parallel(1, omega=0.5)
        mb, mu = o.copy_duals()
        assert np.all(mb + mu <= 1e-12)


def test_fig2_worked_example():
    """Sec. 6, Figure 2: the split of Figure 1's BDD has two pieces and three copy-arc pairs, in
    the arcs the figure draws; the figure's marked path (x1 = 0, x3 = 1, x7 = 0) crosses the cut
    through the pair it marks, so with that pair's duals made cheap the piece energies add up to
    the path's cost."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig2_split.json")))
    fig1 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig1_bdd.json")))["row"]
    n = fig1["n"]
    inst = _from_rows("fig1", n, [(np.array(fig1["cols"]), np.array(fig1["vals"]), fig1["b"], fig1["sense"])],
                      np.zeros(n, np.float32))
    o = Oracle(inst)
    assert o.split([g["cut_place"]]) == 2
    assert o.npairs == len(g["pair_heads"])
    can = o.canonical()
    want_lo = [v for p in g["pieces"] for lay in p["layers"] for v in lay["lo"]]
    want_hi = [v for p in g["pieces"] for lay in p["layers"] for v in lay["hi"]]
    np.testing.assert_array_equal(can["lo"], want_lo)
    np.testing.assert_array_equal(can["hi"], want_hi)
    np.testing.assert_array_equal(can["bdd_depth"], [len(p["layers"]) for p in g["pieces"]])
    np.testing.assert_array_equal(can["occ_var"], [lay["var"] for p in g["pieces"] for lay in p["layers"]])
    # only the marked pair (abar_2, a_2) is cheap on both sides; lambda charges x3 alone.  The
    # earlier piece's best path is then the figure's x1 = 0, x3 = 1 through abar_2 (cost 1), the
    # later piece's enters through a_2 and takes x7 = 0 (cost 0): the marked paths of Figure 2
    lam = np.zeros(3)
    lam[1] = 1.0
    o.set_state(lam)
    mb = np.full(o.npairs, 5.0)
    mu = np.full(o.npairs, 5.0)
    mb[g["marked_pair"]] = 0.0
    mu[g["marked_pair"]] = 0.0
    o.set_copy_duals(mb, mu)
    E = o.energies()
    np.testing.assert_allclose(E, [1.0, 0.0], rtol=0, atol=1e-12)
    # a dearer marked pair moves both energies by its duals: the path is still the only cheap one
    mb[g["marked_pair"]] = 0.5
    mu[g["marked_pair"]] = -0.5
    o.set_copy_duals(mb, mu)
    np.testing.assert_allclose(o.energies(), [1.5, -0.5], rtol=0, atol=1e-12)
