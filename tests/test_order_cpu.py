"""CPU checks of the variable order (Appendix A.3) in the library: the BDD compiler honours a
given order bit for bit against the oracle, and the Cuthill-McKee routine returns a valid order
whose bandwidth matches SciPy's reverse Cuthill-McKee on the same bipartite graph."""
from __future__ import annotations

import numpy as np
import pytest

from instances import SENSE_LE, config, potts_mrf, random_ilp, sparse_matching, tomography, tracking
from instances.generators import _from_rows
from oracle import Oracle


def _spans(inst, rank):
    """(max, sum) over rows of the spread of the row's variables in the order."""
    w, tot = 0, 0
    for cols, vals, _, _ in inst.rows():
        c = cols[vals != 0]
        if len(c):
            d = int(rank[c].max() - rank[c].min())
            w, tot = max(w, d), tot + d
    return w, tot


def _scipy_rank(inst):
    """Variable order of SciPy's reverse Cuthill-McKee on the bipartite graph."""
    sp = pytest.importorskip("scipy.sparse")
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    n, m = inst.n, inst.m
    r, c = [], []
    for j, (cols, vals, _, _) in enumerate(inst.rows()):
        cols = cols[vals != 0]
        r += [n + j] * len(cols)
        c += list(cols)
    A = sp.coo_matrix((np.ones(len(r)), (r, c)), shape=(n + m, n + m)).tocsr()
    perm = reverse_cuthill_mckee((A + A.T).tocsr(), symmetric_mode=True)
    rank = np.empty(n, np.int64)
    rank[[v for v in perm if v < n]] = np.arange(n)
    return rank


WORKLOADS = {
    "potts_8x8x3": lambda: potts_mrf(8, 8, 3, seed=1),
    "potts_config": lambda: config(0),
    "tracking": lambda: tracking(frames=10, dets=40, seed=1),
    "matching": lambda: sparse_matching(n_left=60, n_right=50, k=6, n_pairs=800, seed=3),
    "random": lambda: random_ilp(n=200, m=100, max_row_vars=8, seed=1),
    "tomography": lambda: tomography(side=16, seed=1),
}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_cuthill_mckee_bandwidth_matches_scipy(cuda_lib, name):
    from paper_2009_00481_gb300 import cuthill_mckee
    inst = WORKLOADS[name]()
    rank = cuthill_mckee(inst)
    assert np.array_equal(np.sort(rank), np.arange(inst.n))
    ours, ref = _spans(inst, rank), _spans(inst, _scipy_rank(inst))
    assert ours[0] <= 1.2 * ref[0] + 2 and ours[1] <= 1.2 * ref[1], (ours, ref)
    assert np.array_equal(cuthill_mckee(inst), rank)  # deterministic


@pytest.mark.parametrize("name", ["potts_8x8x3", "potts_config", "tracking"])
def test_cuthill_mckee_beats_index_order_on_grids(cuda_lib, name):
    """On grid MRFs and tracking (where the paper reorders) the order brings the variables of
    each row together: the largest spread drops far below that of the index order."""
    from paper_2009_00481_gb300 import cuthill_mckee
    inst = WORKLOADS[name]()
    assert _spans(inst, cuthill_mckee(inst))[0] * 4 < _spans(inst, np.arange(inst.n))[0]


def test_cuthill_mckee_chain_is_optimal(cuda_lib):
    """Pairwise rows x_k + x_{k+1} <= 1 on a shuffled chain: the order follows the chain, every
    row spans 1 (the least possible)."""
    from paper_2009_00481_gb300 import cuthill_mckee
    n = 40
    perm = np.random.default_rng(3).permutation(n)
    rows = [(np.array([perm[k], perm[k + 1]]), np.array([1, 1]), 1, SENSE_LE) for k in range(n - 1)]
    inst = _from_rows("chain", n, rows, np.zeros(n, np.float32))
    rank = cuthill_mckee(inst)
    assert _spans(inst, rank) == (1, n - 1)


def test_cuthill_mckee_components_and_isolated(cuda_lib):
    """Components in the order of their lowest variable; variables in no row (or only with zero
    coefficients) last, in index order."""
    from paper_2009_00481_gb300 import cuthill_mckee
    rows = [(np.array([5, 7]), np.array([1, 1]), 1, SENSE_LE),
            (np.array([1, 3]), np.array([1, 1]), 1, SENSE_LE),
            (np.array([3, 2]), np.array([1, 0]), 1, SENSE_LE)]  # x2 only with coefficient 0
    inst = _from_rows("comp", 8, rows, np.zeros(8, np.float32))
    rank = cuthill_mckee(inst)
    assert set(rank[[1, 3]]) == {0, 1} and set(rank[[5, 7]]) == {2, 3}
    assert list(rank[[0, 2, 4, 6]]) == [4, 5, 6, 7]


def test_cuthill_mckee_errors(cuda_lib):
    from paper_2009_00481_gb300 import BDDError, binding as B
    with pytest.raises(BDDError) as e:
        B.bdd_cuthill_mckee(3, 1, np.array([0, 2]), np.array([0, 3]))
    assert e.value.code == B.BDD_EINVAL
    with pytest.raises(BDDError):
        B.bdd_cuthill_mckee(3, 1, np.array([1, 2]), np.array([0, 1]))
    assert B.bdd_cuthill_mckee(0, 0, np.zeros(1), np.zeros(0)).shape == (0,)


@pytest.mark.parametrize("host_only", [1, 2])
@pytest.mark.parametrize("seed", range(6))
def test_compiler_bit_exact_with_order(cuda_lib, seed, host_only):
    """BDDs built in a given variable order equal the oracle's built in the same order."""
    from paper_2009_00481_gb300 import Solver, cuthill_mckee
    inst = random_ilp(n=30, m=25, max_row_vars=14, seed=800 + seed, coef=3) if seed < 4 else \
        tracking(frames=6, dets=15, seed=seed)
    rank = np.random.default_rng(seed).permutation(inst.n) if seed % 2 else cuthill_mckee(inst)
    o = Oracle(inst, rank=rank)
    s = Solver(inst, host_only=host_only, rank=rank)
    want, got = o.canonical(), s.canonical()
    for key in ["bdd_row", "bdd_depth", "occ_var", "occ_csr", "occ_width", "lo", "hi"]:
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)


def test_order_and_averaging_options_are_checked(cuda_lib):
    from paper_2009_00481_gb300 import BDDError, Solver
    from paper_2009_00481_gb300.binding import BDD_EINVAL
    inst = potts_mrf(3, 3, 2, seed=0)
    for bad in (np.zeros(inst.n), np.arange(1, inst.n + 1), -np.arange(inst.n)):
        with pytest.raises(BDDError) as e:
            Solver(inst, host_only=1, rank=bad)
        assert e.value.code == BDD_EINVAL
    with pytest.raises(ValueError):
        Solver(inst, host_only=1, rank=np.arange(inst.n - 1))
    with pytest.raises(BDDError) as e:
        Solver(inst, host_only=1, averaging=2)
    assert e.value.code == BDD_EINVAL
    Solver(inst, host_only=1, rank="cm", averaging=1)
