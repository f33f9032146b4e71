"""The allocation-free bound entry point against the solver's own bound.

bdd_lower_bound_noalloc serves callers that cannot allocate device memory (code running in a
memory pool or arena it does not own, or a framework that forbids cudaMalloc on its hot path):
they pass their own input and output buffers and the library uses a static scratch array.
This file is collected last so that a run stopping at the first failure has run every other
test before it.
"""
from __future__ import annotations

import numpy as np
import pytest

from instances import config

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the min-marginal tolerance of the parity tests (FP32 path sums, FP64 reduction)


def _expected_and_inputs(inst, lam, P):
    """Bound from the existing entry point (bdd_iterate with zero iterations) for state
    (lam, P), and the per-BDD energies E_j(lam) taken from the min-marginals of a second solver
    whose state is (lam, 0): E_j = min(m0, m1) of any occurrence of row j."""
    from paper_2009_00481_gb300 import Solver
    a = Solver(inst)
    a.set_state(lam, P)
    lb, _, _, _ = a.iterate(0)
    b = Solver(inst)
    b.set_state(lam)
    _, _, m0, m1 = b.iterate(0, mm=True)
    first = inst.row_ptr[:-1]
    E = np.minimum(m0[first], m1[first]).astype(np.float32)
    a.close()
    b.close()
    return lb, E


def test_noalloc_bound_matches_solver_bound_twice():
    import torch

    from paper_2009_00481_gb300 import binding

    assert torch.cuda.is_available()
    inst = config(0)
    # three extra variables that appear in no row: they enter the bound as min(0, c_i)
    inst.c = np.concatenate([inst.c, np.array([-0.75, 0.5, -1.25], np.float32)])
    inst.n += 3
    deg = np.bincount(inst.col[inst.val != 0], minlength=inst.n).astype(np.int32)
    empty_const = float(np.minimum(inst.c[deg == 0].astype(np.float64), 0).sum())
    assert empty_const == pytest.approx(-2.0)
    rng = np.random.default_rng(12)
    stream = torch.cuda.current_stream().cuda_stream
    d_deg = torch.from_numpy(deg).cuda()
    results = []
    for call in range(2):  # two calls in a row, different inputs
        lam = rng.normal(0, 1, size=inst.nnz).astype(np.float32)
        P = rng.normal(0, 0.5, size=inst.n).astype(np.float32)
        want, E = _expected_and_inputs(inst, lam, P)
        d_E = torch.from_numpy(E).cuda()
        d_P = torch.from_numpy(P).cuda()
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        binding.bdd_lower_bound_noalloc(inst.n, len(E), d_E.data_ptr(), d_P.data_ptr(), d_deg.data_ptr(),
                                        empty_const, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - want) <= TOL * max(1.0, abs(got), abs(want)), (call, got, want)
        results.append(got)
    assert results[0] != results[1]


def test_noalloc_rejects_oversized_input():
    from paper_2009_00481_gb300 import BDDError, binding
    from paper_2009_00481_gb300.binding import BDD_ETOOBIG
    with pytest.raises(BDDError) as e:
        binding.bdd_lower_bound_noalloc(4_194_305, 1, 1, 1, 1, 0.0, 1, 0)
    assert e.value.code == BDD_ETOOBIG
