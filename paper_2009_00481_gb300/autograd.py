"""The smoothed bound as a differentiable PyTorch function of the costs.

``smoothed_bound(c, solver, K)`` returns the smoothed (Appendix A.5) lower bound after K
iterations started from lambda = c/|J_i|, as a float64 CUDA scalar.  Its backward runs the
library's hand-written adjoint kernels (bdd_smooth_backward).  Marshalling only.
"""
from __future__ import annotations

import torch

from . import binding as B


def _stream_ptr():
    s = torch.cuda.current_stream().cuda_stream
    return s if s != 0 else 1  # 1: the legacy default stream PyTorch reports as 0


class SmoothedBound(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, solver, K):
        if not c.is_cuda:
            raise ValueError("costs must be a CUDA tensor")
        c32 = c.detach().to(torch.float32).contiguous()
        bound = torch.empty((), dtype=torch.float64, device=c.device)
        ctx.generation = B.bdd_smooth_forward(solver.h, K, c32.data_ptr(), bound.data_ptr(), _stream_ptr())
        ctx.solver = solver
        ctx.c_dtype = c.dtype
        ctx.keep = c32
        return bound

    @staticmethod
    def backward(ctx, g):
        g64 = g.detach().to(torch.float64).contiguous().reshape(())
        grad = torch.empty(ctx.keep.shape, dtype=torch.float32, device=ctx.keep.device)
        # the checkpoints must still be this forward's (a later forward on the same solver
        # replaces them: the library then refuses with BDD_ESTATE)
        B.bdd_smooth_backward(ctx.solver.h, ctx.generation, g64.data_ptr(), grad.data_ptr(), _stream_ptr())
        return grad.to(ctx.c_dtype), None, None


def smoothed_bound(c: torch.Tensor, solver, K: int) -> torch.Tensor:
    """Smoothed bound after K iterations as a function of the costs c (CUDA tensor [n])."""
    return SmoothedBound.apply(c, solver, K)
