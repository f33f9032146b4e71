"""GPU parity of the variable order (Appendix A.3) and of SRMP averaging (Appendix A.4) against
the FP64 oracle run in the same order with the same averaging.  Tolerances as in the main parity
tests: bound traces 1e-4, min-marginals of the same multipliers 1e-5 (relative, floor 1)."""
from __future__ import annotations

import numpy as np
import pytest

from instances import config, potts_mrf, random_ilp, sparse_matching, tomography, tracking
from oracle import Oracle
from tests.test_gpu_parity import LB_TOL, MM_TOL, MONO_TOL, _trace, close

pytestmark = pytest.mark.gpu

CASES = {
    "potts_20x20x3": lambda: config(0),
    "matching_small": lambda: sparse_matching(n_left=60, n_right=50, k=6, n_pairs=800, seed=3),
    "tomography_16": lambda: tomography(side=16, seed=1, unary_sigma=0.05),
    "tracking_10x40": lambda: tracking(frames=10, dets=40, seed=1),
    "random_wide": lambda: random_ilp(n=60, m=40, max_row_vars=16, seed=11, coef=3),
}


@pytest.fixture(scope="module")
def lib(cuda_lib):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return cuda_lib


def _rank(inst, kind):
    from paper_2009_00481_gb300 import cuthill_mckee
    if kind == "index":
        return None
    if kind == "cm":
        return cuthill_mckee(inst)
    return np.random.default_rng(4).permutation(inst.n)


def _oracle(inst, rank, srmp):
    o = Oracle(inst, rank=rank)
    if srmp:
        o.set_srmp()
    return o


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("averaging", [0, 1])
@pytest.mark.parametrize("order", ["index", "cm", "random"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_trace_parity(lib, name, order, averaging, schedule):
    from paper_2009_00481_gb300 import Solver
    inst = CASES[name]()
    rank = _rank(inst, order)
    iters = 100
    want = _oracle(inst, rank, averaging).run_parallel(iters, omega=0.5)
    got = _trace(Solver(inst, rank=rank, averaging=averaging, schedule=schedule), iters)
    close(got[-1:], want[-1:], LB_TOL)
    close(got[:10], want[:10], LB_TOL)
    assert np.all(np.diff(got) >= -MONO_TOL * np.maximum(1.0, np.abs(got[1:])))


@pytest.mark.parametrize("name", ["matching_small", "tracking_10x40", "random_wide"])
def test_srmp_state_and_folded_outputs(lib, name):
    """After 60 SRMP iterations: pending sums per variable, multipliers folded with the forward
    sweep's shares, and min-marginals of that point match the oracle; the folded multipliers of
    each variable still sum to c_i."""
    from paper_2009_00481_gb300 import Solver
    inst = CASES[name]()
    rank = _rank(inst, "cm")
    s = Solver(inst, rank=rank, averaging=1)
    lb, lam, m0, m1 = s.iterate(60, lam=True, mm=True)
    o = _oracle(inst, rank, True)
    tr = o.run_parallel(60, omega=0.5)
    close([lb], [tr[-1]], LB_TOL)
    _, P = s.get_state()
    close(P, o.pending(), 2e-4)
    close(lam, o.lam(fold=True), 2e-4)
    e0, e1 = o.min_marginals(fold=True)
    close(m0, e0, 5e-4)
    close(m1, e1, 5e-4)
    sums = np.zeros(inst.n)
    np.add.at(sums, inst.col, lam.astype(np.float64))
    deg = np.bincount(inst.col[inst.val != 0], minlength=inst.n)
    close(sums[deg > 0], inst.c[deg > 0], 1e-5)


def test_srmp_same_state_min_marginals(lib):
    """set_state with pending sums prepares the forward sweep's SRMP shares: the folded outputs
    of the same (lambda, P) equal the oracle's."""
    from paper_2009_00481_gb300 import Solver
    inst = CASES["random_wide"]()
    rng = np.random.default_rng(8)
    lam = rng.normal(0, 1, size=inst.nnz).astype(np.float32)
    P = rng.normal(0, 0.5, size=inst.n).astype(np.float32)
    rank = _rank(inst, "random")
    s = Solver(inst, rank=rank, averaging=1)
    s.set_state(lam, P)
    lb, lam_out, m0, m1 = s.iterate(0, lam=True, mm=True)
    o = _oracle(inst, rank, True)
    o.set_state(lam.astype(np.float64), P.astype(np.float64))
    close(lam_out, o.lam(fold=True), 1e-6)
    e0, e1 = o.min_marginals(fold=True)
    close(m0, e0, MM_TOL)
    close(m1, e1, MM_TOL)
    close([lb], [o.bound()], MM_TOL)


@pytest.mark.parametrize("name", ["potts_20x20x3", "tomography_16", "random_wide"])
def test_srmp_schedules_agree(lib, name):
    """Persistent kernel and per-phase kernels run the same SRMP arithmetic bit for bit."""
    from paper_2009_00481_gb300 import Solver
    inst = CASES[name]()
    a = Solver(inst, schedule=0, averaging=1, rank="cm")
    b = Solver(inst, schedule=1, averaging=1, rank="cm")
    close(_trace(a, 30), _trace(b, 30), 1e-12)
    la, pa = a.get_state()
    lb_, pb = b.get_state()
    np.testing.assert_array_equal(la, lb_)
    np.testing.assert_array_equal(pa, pb)


def test_order_leaves_default_averaging_outputs_in_csr_order(lib):
    """The order changes the BDDs' layer order only: with the index order given explicitly the
    run is bit-identical to the default, and outputs stay in CSR positions for any order."""
    from paper_2009_00481_gb300 import Solver
    inst = CASES["tracking_10x40"]()
    a = Solver(inst)
    b = Solver(inst, rank=np.arange(inst.n))
    np.testing.assert_array_equal(_trace(a, 20), _trace(b, 20))
    c = Solver(inst, rank="cm")
    lb, lam, _, _ = c.iterate(20, lam=True)
    o = Oracle(inst, rank=c.rank)
    o.run_parallel(20, omega=0.5)
    close(lam, o.lam(fold=True), 2e-4)


@pytest.mark.parametrize("alpha", [0.1, 0.5])
def test_smoothed_srmp_trace_and_gradient(lib, alpha):
    """Smoothing with SRMP averaging in a Cuthill-McKee order: bound trace against the oracle and
    the gradient against FP64 central differences of the oracle's smoothed bound."""
    import copy

    import torch
    from paper_2009_00481_gb300 import Solver, smoothed_bound
    inst = tracking(frames=5, dets=20, seed=0)
    K = 40
    s = Solver(inst, alpha=alpha, averaging=1, rank="cm")
    rank = s.rank
    o = _oracle(inst, rank, True)
    o.set_alpha(alpha)
    o.set_srmp()
    want = o.run_parallel(K, omega=0.5)
    close(_trace(Solver(inst, alpha=alpha, averaging=1, rank=rank), K), want, LB_TOL)

    def oracle_bound(c):
        j = copy.copy(inst)
        j.c = np.asarray(c, np.float64)
        q = Oracle(j, rank=rank)
        q.set_alpha(alpha)
        q.set_srmp()
        return float(q.run_parallel(K, omega=0.5)[-1])

    c = inst.c.astype(np.float64)
    ct = torch.tensor(c.astype(np.float32), device="cuda", requires_grad=True)
    val = smoothed_bound(ct, s, K)
    val.backward()
    torch.cuda.synchronize()
    close([float(val.item())], [want[-1]], LB_TOL)
    grad = ct.grad.detach().cpu().numpy().astype(np.float64)
    idx = np.random.default_rng(0).choice(inst.n, size=24, replace=False)
    h = 1e-4
    fd = np.array([(oracle_bound(c + h * np.eye(1, inst.n, i)[0]) -
                    oracle_bound(c - h * np.eye(1, inst.n, i)[0])) / (2 * h) for i in idx])
    err = np.abs(grad[idx] - fd) / max(1.0, np.abs(fd).max())
    assert err.max() < 5e-3, err.max()
