"""Planted mistakes: copies of oracle.c with one plausible error each must fail the pins.

Each mutant is a textual edit of a copy of the oracle source, compiled on the CPU into a
temporary directory; the original oracle is untouched.
"""
from __future__ import annotations

import os
import subprocess

import numpy as np
import pytest

from instances import SENSE_EQ, SENSE_GE, SENSE_LE, random_ilp
from instances.generators import _from_rows
from oracle import Oracle, OracleError, load_variant
from tests import bruteforce as bf

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")

MUTANTS = {
    # min-marginal difference with the wrong sign
    "sign": ("return (isinf(m0) || isinf(m1)) ? 0.0 : m1 - m0;",
             "return (isinf(m0) || isinf(m1)) ? 0.0 : m0 - m1;"),
    # deferred averaging share never applied in the forward sweep
    "drop_share": ("        }\n      }\n      h->lam[o] += h->oshare[o];",
                   "        }\n      }\n"),
    # forward update step charges the 1-arc with the wrong layer's multiplier
    "fwd_index": ("            double x = h->fm[u] + h->lam[o - 1];\n            h->fm[v] = agg(h, h->fm[v], x);",
                  "            double x = h->fm[u] + h->lam[o];\n            h->fm[v] = agg(h, h->fm[v], x);"),
    # BDD builder swaps the 0- and 1-successor
    "swap_arcs": ("iv_push(&Llo[l], c0) || iv_push(&Lhi[l], c1)",
                  "iv_push(&Llo[l], c1) || iv_push(&Lhi[l], c0)"),
    # backward step drops the 1-arc cost
    "bwd_theta": ("double a1 = lam_o + bval(h, bm, o, h->hi[u]);",
                  "double a1 = bval(h, bm, o, h->hi[u]);"),
    # bound forgets the slack term of the y-variables
    "bound_slack": ("  for (int b = 0; b < h->nb; ++b) lb += piece_energy(h, b, h->bm);\n  for (int i = 0; i < h->n; ++i)\n    if (h->deg[i] > 0) lb += agg(h, 0.0, h->P[i]);",
                    "  for (int b = 0; b < h->nb; ++b) lb += piece_energy(h, b, h->bm);"),
    # SRMP sets of the forward and backward passes swapped (Appendix A.4)
    "srmp_direction": ("return forward ? l < k - 1 : l > 0;", "return forward ? l > 0 : l < k - 1;"),
    # SRMP without the fallback to all of J_i when J_i^> (J_i^<) is empty
    "srmp_no_fallback": ("if (!h->srmp || cnt == 0)", "if (!h->srmp)"),
    # sequential schedule visits variables in index order whatever the variable order
    "order_visit": ("visit_variable(h, h->order[k], 1, check, m0s, m1s)",
                    "visit_variable(h, k, 1, check, m0s, m1s)"),
    # BDD layers in index order whatever the variable order
    "order_layers": ("long long rx = g_rank ? g_rank[x->col] : x->col, ry = g_rank ? g_rank[y->col] : y->col;",
                     "long long rx = x->col, ry = y->col;"),
}

# planted mistakes in the sub-BDD code (Sec. 6), caught by the split battery
SPLIT_MUTANTS = {
    # copy-arc update with the wrong sign of delta_fwd
    "split_sign": ("h->mu_bar[k] += -h->gamma * h->dfwd[k] + h->gamma * h->dbwd[k];",
                   "h->mu_bar[k] += h->gamma * h->dfwd[k] + h->gamma * h->dbwd[k];"),
    # later pieces start every root at 0 instead of min mu over the entry arcs
    "split_root": ("static double root_msg(const oracle_t *h, long long v) { return h->root_f ? h->root_f[v] : 0.0; }",
                   "static double root_msg(const oracle_t *h, long long v) { (void)v; return h->root_f ? 0.0 : 0.0; }"),
    # copy arcs into top without their dual
    "split_copy_cost": ("if (t <= ORC_COPY0) return h->mu_bar[ORC_COPY0 - t];", "if (t <= ORC_COPY0) return 0.0;"),
    # entry marginal from the forward instead of the backward message of the head
    "split_entry": ("return h->mu[k] + h->bm[h->pair_w[k]];", "return h->mu[k] + h->fm[h->pair_w[k]];"),
    # depth split with floor(k / D) pieces instead of ceil(k / D)
    "split_depth_floor": ("int q = (k + D - 1) / D;", "int q = k / D;"),
}
# planted mistakes in the reverse-mode gradient of the smoothed bound, caught by the gradient
# battery (central differences and the Gibbs marginals at zero iterations)
GRAD_MUTANTS = {
    # the 1-arc multiplier of the previous layer gets no adjoint from the forward messages
    "grad_fwd_theta": ("                glam[ol] += wt;  /* adjoint of lam1 of the previous layer (processed next) */\n",
                       "\n"),
    # d = omega (m1 - m0) reversed with the wrong sign
    "grad_sign": ("double g1 = omega * gd, g0 = -omega * gd;", "double g1 = -omega * gd, g0 = omega * gd;"),
    # the share weight 1/|J_i| dropped on the way back to the pending sums
    "grad_share": ("gP[h->occ_var[o]] += w[o] * gshr[o];", "gP[h->occ_var[o]] += gshr[o];"),
    # lambda_0 = c_i / |J_i| reversed without the division
    "grad_init": ("grad_c[h->occ_var[o]] += glam[o] / (double)h->deg[h->occ_var[o]];",
                  "grad_c[h->occ_var[o]] += glam[o];"),
    # the recorded deltas get no adjoint from the pending sums they form
    "grad_pending": ("gdel[h->var_occ[t]] += gP[i];", "(void)t;"),
}
MUTANTS_ALL = {**MUTANTS, **SPLIT_MUTANTS, **GRAD_MUTANTS}


def _compile(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTANTS_ALL[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(path), "-lm"])
    return load_variant(str(so))


def _pins_hold(lib) -> bool:
    """A compact battery of the pins: enumeration of BDDs and min-marginals, the parallel
    schedule's checks, and weak duality against brute force."""
    rng = np.random.default_rng(7)
    for t in range(12):
        k = int(rng.integers(2, 9))
        vals = rng.integers(1, 4, size=k) * rng.choice([-1, 1], size=k)
        sense = [SENSE_LE, SENSE_EQ, SENSE_GE][t % 3]
        x0 = rng.integers(0, 2, size=k)
        b = int(vals @ x0)
        lam = rng.normal(size=k)
        inst = _from_rows("r", k, [(np.arange(k), vals, b, sense)], np.zeros(k, np.float32))
        try:
            o = Oracle(inst, lib=lib)
        except OracleError:
            return False
        layers = bf.split_bdds(o.canonical())[0]
        feas = bf.row_feasible(vals, b, sense)
        acc = np.array([bf.walk(layers, x)[0] for x in bf.assignments(k)])
        if not np.array_equal(acc, feas):
            return False
        o.set_state(lam)
        m0, m1 = o.min_marginals(fold=False)
        em0, em1, _, _ = bf.min_marginals_enum(vals, b, sense, lam)
        if not (np.allclose(m0, em0, atol=1e-12) and np.allclose(m1, em1, atol=1e-12)):
            return False
    for seed in range(3):
        inst = random_ilp(n=14, m=10, max_row_vars=6, seed=500 + seed)
        opt = bf.ilp_optimum(inst)
        o = Oracle(inst, lib=lib)
        tr = o.run_parallel(15, omega=0.5, check=True)
        w = o.worst()
        if w["incremental_mm"] > 1e-10 or w["invariant"] > 1e-12 or w["monotone_drop"] > 1e-12:
            return False
        if tr.max() > opt + 1e-9:
            return False
    # variable order and SRMP: both schedules against enumeration (Appendix A.3, A.4)
    for seed in range(2):
        inst = random_ilp(n=9, m=6, max_row_vars=5, seed=520 + seed)
        rank = np.random.default_rng(seed).permutation(inst.n)
        for srmp in (False, True):
            o = Oracle(inst, lib=lib, rank=rank)
            if srmp:
                o.set_srmp()
            if not np.allclose(o.run_sequential(3), bf.sequential_enum(inst, 3, rank, srmp),
                               rtol=0, atol=1e-10):
                return False
            o.reset()
            if not np.allclose(o.run_parallel(4, omega=0.5),
                               bf.parallel_enum(inst, 4, 0.5, rank, srmp), rtol=0, atol=1e-10):
                return False
    return True


def _split_pins_hold(lib) -> bool:
    """Piece energies by enumeration with random duals, and the split schedule's checks."""
    from tests.test_oracle_split import _piece_energies_enum
    rng = np.random.default_rng(3)
    for t in range(6):
        k = int(rng.integers(5, 10))
        vals = rng.integers(1, 4, size=k) * rng.choice([-1, 1], size=k)
        sense = [SENSE_LE, SENSE_EQ, SENSE_GE][t % 3]
        b = int(vals @ rng.integers(0, 2, size=k))
        inst = _from_rows("r", k, [(np.arange(k), vals, b, sense)], np.zeros(k, np.float32))
        layers = bf.split_bdds(Oracle(inst, lib=lib).canonical())[0]
        cuts = sorted(rng.choice(np.arange(1, k), size=2, replace=False).tolist())
        o = Oracle(inst, lib=lib)
        o.split(cuts)
        lam = rng.normal(size=k)
        o.set_state(lam)
        mb, mu = rng.normal(size=o.npairs), rng.normal(size=o.npairs)
        o.set_copy_duals(mb, mu)
        want = _piece_energies_enum(vals, b, sense, lam, cuts, mb, mu, layers)
        if not np.allclose(o.energies(), want, rtol=0, atol=1e-12):
            return False
    for seed in range(3):
        inst = random_ilp(n=15, m=10, max_row_vars=9, seed=40 + seed)
        o = Oracle(inst, lib=lib)
        o.split([5, 10])
        tr = o.run_parallel(30, omega=0.5, check=True)
        w = o.worst()
        if w["incremental_mm"] > 1e-10 or w["invariant"] > 1e-12 or w["monotone_drop"] > 1e-12:
            return False
        mb, mu = o.copy_duals()
        if np.any(mb + mu > 1e-12) or tr.max() > bf.ilp_optimum(inst) + 1e-9:
            return False
    for D in (2, 3):  # depth split: no piece deeper than D, every piece an honest subproblem
        inst = random_ilp(n=20, m=12, max_row_vars=11, seed=70 + D, coef=3)
        o = Oracle(inst, lib=lib)
        o.split_depth(D)
        if o.canonical()["bdd_depth"].max() > D:
            return False
        tr = o.run_parallel(20, omega=0.5, check=True)
        w = o.worst()
        if w["incremental_mm"] > 1e-10 or w["monotone_drop"] > 1e-12 or tr.max() > bf.ilp_optimum(inst) + 1e-9:
            return False
    return True


def test_original_passes_split_battery():
    from oracle import _load
    assert _split_pins_hold(_load())


@pytest.mark.parametrize("name", sorted(SPLIT_MUTANTS))
def test_split_mutant_is_caught(tmp_path, name):
    lib = _compile(tmp_path, name)
    assert not _split_pins_hold(lib), f"planted mistake '{name}' passed every split pin"


def test_original_passes_battery():
    from oracle import _load
    assert _pins_hold(_load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    lib = _compile(tmp_path, name)
    assert not _pins_hold(lib), f"planted mistake '{name}' passed every pin"


def _grad_pins_hold(lib) -> bool:
    """The gradient battery of tests/test_oracle_smooth.py on small cases: every coordinate
    against central differences, and the Gibbs marginals at zero iterations."""
    from tests.test_oracle_smooth import GRAD_CASES, _central_differences, _oracle_gradient
    for name in ("tracking_3x6", "random_ilp"):
        inst = GRAD_CASES[name]()
        for K, srmp in ((1, False), (4, True)):
            _, g = _oracle_gradient(inst, 0.3, K, srmp, lib=lib)
            fd = _central_differences(inst, 0.3, K, srmp, lib=lib)
            if np.abs(g - fd).max() > 1e-6 * max(1.0, np.abs(fd).max()):
                return False
    return True


def test_original_passes_gradient_battery():
    from oracle import _load
    assert _grad_pins_hold(_load())


@pytest.mark.parametrize("name", sorted(GRAD_MUTANTS))
def test_gradient_mutant_is_caught(tmp_path, name):
    lib = _compile(tmp_path, name)
    assert not _grad_pins_hold(lib), f"planted mistake '{name}' passed every gradient pin"

