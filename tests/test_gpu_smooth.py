"""GPU parity of the smoothed (log-sum-exp) variant (Appendix A.5) against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest

from instances import config, potts_mrf, sparse_matching, tomography, tracking
from oracle import Oracle
from tests.test_gpu_parity import LB_TOL, MM_TOL, _trace, close

pytestmark = pytest.mark.gpu

CASES = {
    "potts_8x8x3": lambda: potts_mrf(8, 8, 3, seed=2),
    "tracking_10x40": lambda: tracking(frames=10, dets=40, seed=1),
    "matching_small": lambda: sparse_matching(n_left=60, n_right=50, k=6, n_pairs=800, seed=3),
    # tomography (the paper smooths its tomography runs, Sec. 7): the 16x16 projections fit warp
    # tiles (up to 25 nodes per layer), the 24x24 ones need block tiles (up to 36)
    "tomography_16": lambda: tomography(side=16, seed=1, unary_sigma=0.05),
    "tomography_24": lambda: tomography(side=24, seed=2, unary_sigma=0.05),
}


@pytest.fixture(scope="module")
def lib(cuda_lib):
    import torch
    assert torch.cuda.is_available()
    return cuda_lib


def solver(inst, **kw):
    from paper_2009_00481_gb300 import Solver
    return Solver(inst, **kw)


@pytest.mark.parametrize("alpha", [0.1, 0.5])
@pytest.mark.parametrize("name", sorted(CASES))
def test_smoothed_trace_parity(lib, name, alpha):
    inst = CASES[name]()
    o = Oracle(inst)
    o.set_alpha(alpha)
    want = o.run_parallel(60, omega=0.5)
    got = _trace(solver(inst, alpha=alpha), 60)
    close(got, want, LB_TOL)  # every iterate


@pytest.mark.parametrize("name", sorted(CASES))
def test_smoothed_marginals_same_lambda(lib, name):
    inst = CASES[name]()
    alpha = 0.2
    rng = np.random.default_rng(9)
    lam = rng.normal(0, 1, size=inst.nnz).astype(np.float32)
    s = solver(inst, alpha=alpha)
    s.set_state(lam)
    lb, _, m0, m1 = s.iterate(0, mm=True)
    o = Oracle(inst)
    o.set_alpha(alpha)
    o.set_state(lam.astype(np.float64))
    e0, e1 = o.min_marginals(fold=True)
    close(m0, e0, MM_TOL)
    close(m1, e1, MM_TOL)
    close([lb], [o.bound()], MM_TOL)


def test_small_alpha_recovers_min_sum(lib):
    inst = config(0)
    plain = _trace(solver(inst), 40)
    soft = _trace(solver(inst, alpha=1e-5), 40)
    close(soft, plain, LB_TOL)


def test_smoothing_block_tiles_and_width_limit(lib):
    """Smoothed solvers run block tiles of at most 128 nodes per layer (tomography projections);
    a row with layers over 128 nodes is refused."""
    from paper_2009_00481_gb300 import BDDError
    from paper_2009_00481_gb300.binding import BDD_ETOOBIG
    from tests.test_gpu_parity import _wide_rows_instance
    s = solver(tomography(side=32, seed=1), alpha=0.1)
    assert s.block_tiles > 0 and 32 < s.max_width <= 128
    with pytest.raises(BDDError) as e:
        solver(_wide_rows_instance(), alpha=0.1)
    assert e.value.code == BDD_ETOOBIG


def test_smoothed_marginals_same_lambda_full_tomography(lib):
    """Same-multiplier smoothed marginals on the full 64x64 tomography (block tiles of 33..97
    nodes per layer), element by element."""
    inst = config(2)
    alpha = 0.05
    rng = np.random.default_rng(4)
    lam = rng.normal(0, 1, size=inst.nnz).astype(np.float32)
    lam[inst.val == 0] = 0
    P = rng.normal(0, 0.5, size=inst.n).astype(np.float32)
    s = solver(inst, alpha=alpha)
    assert s.block_tiles > 0
    s.set_state(lam, P)
    lb, _, m0, m1 = s.iterate(0, mm=True)
    o = Oracle(inst)
    o.set_alpha(alpha)
    o.set_state(lam.astype(np.float64), P.astype(np.float64))
    e0, e1 = o.min_marginals(fold=True)
    close(m0, e0, MM_TOL)
    close(m1, e1, MM_TOL)
    close([lb], [o.bound()], MM_TOL)


@pytest.mark.parametrize("alpha", [0.1, 0.5])
def test_gradient_block_tiles_matches_oracle_gradient(lib, alpha):
    """The adjoint of block tiles: d(bound)/dc after K = 20 smoothed iterations on a 24x24
    tomography with unary costs (projection layers up to 36 nodes wide), every coordinate
    against the oracle's FP64 reverse-mode gradient."""
    inst = tomography(side=24, seed=2, unary_sigma=0.2)
    K = 20
    s0 = solver(inst, alpha=alpha)
    assert s0.block_tiles > 0
    val, grad, _ = _gpu_value_and_grad(inst, inst.c.astype(np.float64), alpha, K)
    o = Oracle(inst)
    o.set_alpha(alpha)
    want_val, want = o.smooth_gradient(K, omega=0.5)
    close([val], [want_val], LB_TOL)
    scale = max(1.0, np.abs(want).max())
    err = np.abs(grad - want) / scale
    assert err.max() <= 1e-4, err.max()


# ------------------------------------------------------------------------------------------
# gradient of the smoothed bound (hand-written adjoints) against FP64 central differences
# ------------------------------------------------------------------------------------------

def _oracle_smoothed_bound(inst, c, alpha, K):
    import copy
    j = copy.copy(inst)
    j.c = np.asarray(c, np.float64)
    o = Oracle(j)
    o.set_alpha(alpha)
    return float(o.run_parallel(K, omega=0.5)[-1])


def _gpu_value_and_grad(inst, c, alpha, K, **kw):
    import torch
    from paper_2009_00481_gb300 import smoothed_bound
    s = solver(inst, alpha=alpha, **kw)
    ct = torch.tensor(np.asarray(c, np.float32), device="cuda", requires_grad=True)
    val = smoothed_bound(ct, s, K)
    val.backward()
    torch.cuda.synchronize()
    return float(val.item()), ct.grad.detach().cpu().numpy().astype(np.float64), s


@pytest.mark.parametrize("srmp", [False, True])
@pytest.mark.parametrize("alpha", [0.1, 0.5])
def test_gradient_matches_oracle_gradient(lib, alpha, srmp):
    """d(bound)/dc of the smoothed bound after K = 50 iterations on the 5-frame x 20-detection
    tracking slice: every coordinate of the GPU adjoint (FP32) against the oracle's FP64
    reverse-mode gradient (itself pinned against central differences on the CPU), within 1e-4
    of the gradient's scale; the bound value within the bound tolerance."""
    inst = tracking(frames=5, dets=20, seed=0)
    K = 50
    c = inst.c.astype(np.float64)
    kw = {"averaging": 1} if srmp else {}
    val, grad, _ = _gpu_value_and_grad(inst, c, alpha, K, **kw)
    o = Oracle(inst)
    if srmp:
        o.set_srmp(True)
    o.set_alpha(alpha)
    want_val, want = o.smooth_gradient(K, omega=0.5)
    close([val], [want_val], LB_TOL)
    scale = max(1.0, np.abs(want).max())
    err = np.abs(grad - want) / scale
    assert err.max() <= 1e-4, (err.max(), np.c_[np.argsort(-err)[:5], grad[np.argsort(-err)[:5]],
                                                 want[np.argsort(-err)[:5]]])


@pytest.mark.parametrize("name", ["tracking_5x20", "tomography_24"])
def test_gradient_kept_messages_match_recomputed(lib, name):
    """The backward either reads the messages the forward kept or recomputes them from the
    multipliers' checkpoints (bdd_options.smooth_messages): the same bound and the same gradient
    (to 1e-6 of its scale), on warp tiles (tracking) and block tiles (tomography); keeping them
    holds (2K + 1) N more floats of device memory."""
    import torch
    from paper_2009_00481_gb300 import binding as B, smoothed_bound
    inst = tracking(frames=5, dets=20, seed=0) if name == "tracking_5x20" else \
        tomography(side=24, seed=2, unary_sigma=0.2)
    K, alpha = 12, 0.1
    out, grown = {}, {}
    for keep in (0, 1):
        s = solver(inst, alpha=alpha, smooth_messages=keep)
        before = int(B.bdd_sizes(s.h)[8])
        for rep in range(2):  # the second forward reuses the buffers
            ct = torch.tensor(inst.c.astype(np.float32), device="cuda", requires_grad=True)
            val = smoothed_bound(ct, s, K)
            val.backward()
            torch.cuda.synchronize()
            out[keep, rep] = (float(val.item()), ct.grad.detach().cpu().numpy().astype(np.float64))
        grown[keep] = int(B.bdd_sizes(s.h)[8]) - before
        n_nodes = s.N
        s.close()
    extra = grown[1] - grown[0]
    assert 4 * (2 * K + 1) * n_nodes <= extra <= 4 * (2 * K + 1) * n_nodes + 512, (grown, n_nodes)
    (v0, g0), (v1, g1) = out[0, 0], out[1, 0]
    assert v0 == v1
    scale = max(1.0, np.abs(g0).max())
    assert np.abs(g1 - g0).max() <= 1e-6 * scale, np.abs(g1 - g0).max()
    for keep in (0, 1):
        assert out[keep, 1][0] == out[keep, 0][0]
        np.testing.assert_array_equal(out[keep, 1][1], out[keep, 0][1])


@pytest.mark.parametrize("alpha", [0.1, 0.5])
def test_gradient_matches_oracle_central_differences(lib, alpha):
    """The same gradient against FP64 central differences of the oracle's bound on 16 sampled
    coordinates (an independent check of the adjoint that does not go through the oracle's
    reverse mode)."""
    inst = tracking(frames=5, dets=20, seed=0)
    K = 50
    c = inst.c.astype(np.float64)
    _, grad, _ = _gpu_value_and_grad(inst, c, alpha, K)
    rng = np.random.default_rng(0)
    idx = rng.choice(inst.n, size=16, replace=False)
    h = 1e-4
    fd = np.zeros(len(idx))
    for t, i in enumerate(idx):
        cp, cm = c.copy(), c.copy()
        cp[i] += h
        cm[i] -= h
        fd[t] = (_oracle_smoothed_bound(inst, cp, alpha, K) - _oracle_smoothed_bound(inst, cm, alpha, K)) / (2 * h)
    scale = max(1.0, np.abs(fd).max())
    err = np.abs(grad[idx] - fd) / scale
    assert err.max() < 1e-4, (err.max(), np.c_[idx, grad[idx], fd][np.argsort(-err)[:5]])


def test_gradient_directional_derivative(lib):
    """The full gradient against a GPU directional difference along a random direction."""
    inst = potts_mrf(6, 6, 3, seed=5)
    alpha, K = 0.2, 20
    c = inst.c.astype(np.float64)
    val, grad, _ = _gpu_value_and_grad(inst, c, alpha, K)
    rng = np.random.default_rng(1)
    v = rng.normal(size=inst.n)
    eps = 1e-2
    vp = _oracle_smoothed_bound(inst, c + eps * v, alpha, K)
    vm = _oracle_smoothed_bound(inst, c - eps * v, alpha, K)
    dd = (vp - vm) / (2 * eps)
    assert abs(grad @ v - dd) <= 2e-3 * max(1.0, abs(dd), np.abs(grad) @ np.abs(v))


def test_smoothed_forward_small_alpha_recovers_min_sum(lib):
    """tau -> 0: the smoothed bound after K iterations tends to the min-sum bound."""
    import torch
    from paper_2009_00481_gb300 import smoothed_bound
    inst = potts_mrf(8, 8, 3, seed=6)
    K = 30
    plain = _trace(solver(inst), K)[-1]
    s = solver(inst, alpha=1e-4)
    ct = torch.tensor(inst.c, device="cuda")
    val = float(smoothed_bound(ct, s, K).item())
    close([val], [plain], LB_TOL)


def test_backward_needs_matching_forward(lib):
    import torch
    from paper_2009_00481_gb300 import BDDError, binding, smoothed_bound
    from paper_2009_00481_gb300.binding import BDD_ESTATE
    inst = potts_mrf(4, 4, 2, seed=1)
    s = solver(inst, alpha=0.3)
    g = torch.ones((), dtype=torch.float64, device="cuda")
    out = torch.zeros(inst.n, dtype=torch.float32, device="cuda")
    with pytest.raises(BDDError) as e:  # no forward yet
        binding.bdd_smooth_backward(s.h, 0, g.data_ptr(), out.data_ptr())
    assert e.value.code == BDD_ESTATE
    ct = torch.tensor(inst.c, device="cuda", requires_grad=True)
    val = smoothed_bound(ct, s, 5)
    s.iterate(1)  # changes the state: the recorded forward is stale
    with pytest.raises(BDDError) as e:
        val.backward()
    assert e.value.code == BDD_ESTATE
    plain = solver(inst)
    with pytest.raises(BDDError) as e:  # min-sum solvers have no smoothed bound
        smoothed_bound(ct, plain, 5)
    assert e.value.code == BDD_ESTATE


def test_two_forwards_then_one_backward_refused(lib):
    """Two smoothed bounds of one solver feeding one loss: the second forward replaces the
    checkpoints, so the first one's backward must be refused rather than return the gradient of
    the second one's trajectory; the second one's backward stays valid."""
    import torch
    from paper_2009_00481_gb300 import BDDError, smoothed_bound
    from paper_2009_00481_gb300.binding import BDD_ESTATE
    inst = potts_mrf(4, 4, 2, seed=1)
    s = solver(inst, alpha=0.3)
    c1 = torch.tensor(inst.c, device="cuda", requires_grad=True)
    c2 = torch.tensor(inst.c * 0.5, device="cuda", requires_grad=True)
    v1 = smoothed_bound(c1, s, 5)
    v2 = smoothed_bound(c2, s, 5)
    v2.backward()
    assert c2.grad is not None and torch.isfinite(c2.grad).all()
    with pytest.raises(BDDError) as e:
        v1.backward()
    assert e.value.code == BDD_ESTATE
    v3 = smoothed_bound(c1, s, 5)
    v4 = smoothed_bound(c2, s, 5)
    with pytest.raises(BDDError) as e:  # both in one loss
        (v3 + v4).backward()
    assert e.value.code == BDD_ESTATE

