"""The checked build of the library (the sweep kernels compiled with -DBDD_CHECKED: every window,
node, occurrence, CSR and BDD index is checked before use, and a failed check records BDD_EDEVICE
instead of touching memory out of bounds) on the parity cases: on valid slabs no check fires,
so every call returns BDD_OK, and the results match the oracle as those of the normal build do.
The cases run in a subprocess that loads the checked library (BDD_DBCA_CHECKED=1); they cover
lane tiles, teams of every staging variant, both block-tile paths, the persistent kernel, the
smoothed sweeps and sub-BDDs."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, ROOT)
from instances import config, potts_mrf, sparse_matching, tomography, tracking, random_ilp, SENSE_LE
from instances.generators import _from_rows
from oracle import Oracle
from paper_2009_00481_gb300 import Solver, binding

assert binding.load()._name.endswith("libbdd_dbca_checked.so"), binding.load()._name

def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    fa, fb = np.isfinite(a), np.isfinite(b)
    if not np.array_equal(fa, fb) or not np.array_equal(a[~fa], b[~fb]):
        return float("inf")  # an infinite min-marginal (a forced variable) on one side only
    a, b = a[fa], b[fb]
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.maximum(np.abs(a), np.abs(b)))))

rng = np.random.default_rng(3)
rows = [(np.arange(300), np.ones(300), 149, SENSE_LE)]
for k in [2, 3, 5, 9, 17, 33, 40]:
    rows.append((np.sort(rng.choice(300, size=k, replace=False)), np.ones(k), k // 2, SENSE_LE))
wide = _from_rows("wide", 300, rows, rng.normal(size=300).astype(np.float32))
cases = {
    "potts": potts_mrf(8, 8, 3, seed=2),
    "matching": sparse_matching(n_left=60, n_right=50, k=6, n_pairs=800, seed=3),
    "tomography": tomography(side=16, seed=1, unary_sigma=0.05),
    "tracking": tracking(frames=6, dets=20, seed=1),
    "wide": wide,
}
variants = [{}, {"lanes": 0}, {"lanes": 0, "staging": 1}, {"lanes": 0, "staging": 2}, {"staging": 2},
            {"schedule": 0}, {"split_depth": 3}]
iters = 30
for name, inst in cases.items():
    o = Oracle(inst)
    want = o.run_parallel(iters, omega=0.5)
    e0, e1 = o.min_marginals(fold=True)
    for kw in variants:
        s = Solver(inst, omega=0.5, **kw)
        lb, lam, m0, m1 = s.iterate(iters, lam=True, mm=True)  # BDDError on a failed check
        if "split_depth" in kw:
            os_ = Oracle(inst)
            os_.split_depth(kw["split_depth"])
            ref = os_.run_parallel(iters, omega=0.5)[-1]
        else:
            ref = want[-1]
            assert rel(m0, e0) < 5e-4 and rel(m1, e1) < 5e-4, (name, kw, rel(m0, e0), rel(m1, e1))
        assert rel([lb], [ref]) < 1e-4, (name, kw, lb, ref)
        s.close()
    if o.max_width <= 32:  # smoothed sweeps (warp tiles)
        so = Oracle(inst)
        so.set_alpha(0.2)
        s = Solver(inst, omega=0.5, alpha=0.2)
        lb, _, _, _ = s.iterate(iters)
        assert rel([lb], [so.run_parallel(iters, omega=0.5)[-1]]) < 1e-4, name
        s.close()
print("checked build: all cases ok")
"""


def test_checked_build_parity_cases(cuda_lib):
    import torch
    assert torch.cuda.is_available()
    env = dict(os.environ, BDD_DBCA_CHECKED="1")
    res = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + SCRIPT], env=env, capture_output=True,
                         text=True, cwd=ROOT, timeout=900)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
    assert "all cases ok" in res.stdout
