"""CPU checks of sub-BDDs in the library (Sec. 6, Def. of sub-BDDs and copy-arcs): the host
split of the canonical BDDs, with the copy arcs encoded as top-terminal codes -4 - k, equals the
oracle's split bit for bit (compiled on the host, and read back from the host copy of the slab
layout); the balanced cut places give intervals of similar node counts; bad split options are
refused."""
from __future__ import annotations

import numpy as np
import pytest

from instances import config, potts_mrf, random_ilp, tomography, tracking
from oracle import Oracle

KEYS = ["bdd_row", "bdd_depth", "occ_var", "occ_csr", "occ_width", "lo", "hi"]

WORKLOADS = {
    "potts_config": lambda: config(0),
    "tomography_12": lambda: tomography(side=12, seed=3, unary_sigma=0.1),
    "tracking": lambda: tracking(frames=6, dets=20, seed=2),
    "random": lambda: random_ilp(n=40, m=30, max_row_vars=14, seed=9, coef=3),
}


def _random_cuts(n, k, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(np.arange(1, n), size=k, replace=False)).astype(np.int32)


@pytest.mark.parametrize("host_only", [1, 2])
@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_split_bit_exact_with_oracle(cuda_lib, name, host_only):
    from paper_2009_00481_gb300 import Solver
    inst = WORKLOADS[name]()
    cuts = _random_cuts(inst.n, 3, seed=len(name))
    o = Oracle(inst)
    nb = o.split(cuts)
    s = Solver(inst, host_only=host_only, cuts=cuts)
    assert (s.nb, s.n_cuts, s.npairs) == (nb, len(cuts), o.npairs)
    assert o.npairs > 0
    np.testing.assert_array_equal(s.cuts(), cuts)
    want, got = o.canonical(), s.canonical()
    for key in KEYS:
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)
    assert (got["lo"] <= -4).sum() + (got["hi"] <= -4).sum() == o.npairs


@pytest.mark.parametrize("seed", range(6))
def test_split_bit_exact_in_a_random_order(cuda_lib, seed):
    """Cut places refer to the variable order in use (Appendix A.3 with Sec. 6)."""
    from paper_2009_00481_gb300 import Solver
    inst = random_ilp(n=30, m=25, max_row_vars=12, seed=300 + seed, coef=3)
    rank = np.random.default_rng(seed).permutation(inst.n).astype(np.int32)
    cuts = _random_cuts(inst.n, 1 + seed % 3, seed)
    o = Oracle(inst, rank=rank)
    o.split(cuts)
    s = Solver(inst, host_only=1 + seed % 2, rank=rank, cuts=cuts)
    want, got = o.canonical(), s.canonical()
    for key in KEYS:
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)


def _nodes_per_place(inst, rank=None):
    """Nodes of each place of the order, from the oracle's canonical (unsplit) BDDs."""
    can = Oracle(inst, rank=rank).canonical()
    at = np.zeros(inst.n, np.int64)
    place = np.arange(inst.n) if rank is None else np.asarray(rank)
    np.add.at(at, place[can["occ_var"]], can["occ_width"])
    return at


@pytest.mark.parametrize("k", [2, 3, 4, 8])
@pytest.mark.parametrize("name", ["potts_config", "tomography_12", "tracking"])
def test_balanced_cuts(cuda_lib, name, k):
    """Every interval holds at most N/k nodes plus one place's nodes, every cut is needed (the
    interval before it holds at least N/k minus one place's nodes in total with all earlier
    ones), and the pieces equal the oracle's split at the same places."""
    from paper_2009_00481_gb300 import Solver
    inst = WORKLOADS[name]()
    s = Solver(inst, host_only=1, split=k)
    cuts = s.cuts()
    assert len(cuts) == s.n_cuts <= k - 1
    assert np.all(np.diff(cuts) > 0) and (len(cuts) == 0 or (cuts[0] >= 1 and cuts[-1] < inst.n))
    at = _nodes_per_place(inst)
    N, big = at.sum(), at.max()
    edges = np.concatenate([[0], cuts, [inst.n]])
    sizes = np.array([at[a:b].sum() for a, b in zip(edges[:-1], edges[1:])])
    assert sizes.sum() == N
    assert np.all(sizes <= N / k + big + 1e-9), (sizes, N / k)
    prefix = np.cumsum(sizes)
    for t in range(len(cuts)):
        assert prefix[t] * k >= (t + 1) * N - k * big, (t, prefix[t], N / k)
    o = Oracle(inst)
    o.split(cuts)
    got = s.canonical()
    for key in KEYS:
        np.testing.assert_array_equal(got[key], o.canonical()[key], err_msg=key)


def test_no_split_for_one_interval(cuda_lib):
    from paper_2009_00481_gb300 import Solver
    inst = potts_mrf(4, 4, 3, seed=0)
    for k in (0, 1):
        s = Solver(inst, host_only=1, split=k)
        assert s.n_cuts == 0 and s.npairs == 0 and s.nb == Oracle(inst).nb


def test_split_option_errors(cuda_lib):
    from paper_2009_00481_gb300 import BDDError, Solver
    from paper_2009_00481_gb300.binding import BDD_EINVAL
    inst = potts_mrf(3, 3, 2, seed=0)
    bad = [dict(cuts=[0]), dict(cuts=[3, 3]), dict(cuts=[5, 2]), dict(cuts=[inst.n]),
           dict(cuts=[2], gamma=0.0), dict(cuts=[2], gamma=1.5), dict(split=-1),
           dict(split=2, alpha=0.1)]
    for kw in bad:
        with pytest.raises(BDDError) as e:
            Solver(inst, host_only=1, **kw)
        assert e.value.code == BDD_EINVAL, kw


@pytest.mark.parametrize("host_only", [1, 2])
@pytest.mark.parametrize("D", [1, 3, 8, 32])
@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_depth_split_bit_exact_with_oracle(cuda_lib, name, D, host_only):
    """Pieces of at most D layers equal the oracle's depth split bit for bit."""
    from paper_2009_00481_gb300 import Solver
    inst = WORKLOADS[name]()
    o = Oracle(inst)
    nb = o.split_depth(D)
    s = Solver(inst, host_only=host_only, split_depth=D)
    assert (s.nb, s.n_cuts, s.npairs, s.split_depth) == (nb, 0, o.npairs, D)
    assert s.max_depth <= D
    want, got = o.canonical(), s.canonical()
    for key in KEYS:
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)


def test_depth_split_full_tomography_shape(cuda_lib):
    """Tomography 64x64x3: projections of up to 128 layers in pieces of at most 32."""
    from paper_2009_00481_gb300 import Solver
    inst = config(2)
    whole = Solver(inst, host_only=1)
    s = Solver(inst, host_only=1, split_depth=32)
    assert whole.max_depth == 128 and s.max_depth == 32 and s.nb > whole.nb and s.npairs > 0
    o = Oracle(inst)
    o.split_depth(32)
    assert (o.nb, o.npairs) == (s.nb, s.npairs)


def test_fig2_worked_example_library(cuda_lib):
    """The library's split of Figure 1's BDD at the cut of Figure 2 (Sec. 6) gives the pieces and
    copy arcs of the golden fixture, bit for bit (host compile and host slab layout)."""
    import json
    import os
    from instances.generators import _from_rows
    from paper_2009_00481_gb300 import Solver
    here = os.path.join(os.path.dirname(__file__), "golden")
    g = json.load(open(os.path.join(here, "fig2_split.json")))
    row = json.load(open(os.path.join(here, "fig1_bdd.json")))["row"]
    n = row["n"]
    inst = _from_rows("fig1", n, [(np.array(row["cols"]), np.array(row["vals"]), row["b"], row["sense"])],
                      np.zeros(n, np.float32))
    for host_only in (1, 2):
        s = Solver(inst, host_only=host_only, cuts=[g["cut_place"]])
        assert (s.nb, s.npairs) == (2, len(g["pair_heads"]))
        can = s.canonical()
        np.testing.assert_array_equal(can["lo"], [v for p in g["pieces"] for lay in p["layers"] for v in lay["lo"]])
        np.testing.assert_array_equal(can["hi"], [v for p in g["pieces"] for lay in p["layers"] for v in lay["hi"]])
        np.testing.assert_array_equal(can["bdd_depth"], [len(p["layers"]) for p in g["pieces"]])


def test_split_abi_errors_on_host(cuda_lib):
    """Calls of the sub-BDD ABI on host-only solvers: cut places readable, copy duals need device
    state (BDD_ESTATE), missing arrays refused (BDD_EINVAL); an unsplit solver reports no cuts
    and no pairs."""
    from paper_2009_00481_gb300 import BDDError, Solver
    from paper_2009_00481_gb300 import binding as B
    inst = WORKLOADS["random"]()
    s = Solver(inst, host_only=1, split=3)
    cuts = s.cuts()
    assert len(cuts) == s.n_cuts >= 1 and s.npairs > 0
    with pytest.raises(BDDError) as e:
        s.copy_duals()
    assert e.value.code == B.BDD_ESTATE
    lib = B.load()
    assert lib.bdd_set_copy_duals(s.h, None, None) == B.BDD_EINVAL
    assert lib.bdd_get_cuts(s.h, None) == B.BDD_EINVAL
    plain = Solver(inst, host_only=1)
    assert plain.n_cuts == 0 and plain.npairs == 0 and plain.split_depth == 0
    assert len(plain.cuts()) == 0
    assert lib.bdd_get_cuts(plain.h, None) == B.BDD_OK
