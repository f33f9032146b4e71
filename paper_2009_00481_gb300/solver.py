"""Convenience wrapper of one solver handle.  Marshalling only; PyTorch (optional) supplies
device buffers and streams for :meth:`Solver.iterate_device`."""
from __future__ import annotations

from . import binding as B

# cudaStreamLegacy: the handle of the legacy default stream that PyTorch's default stream
# reports as 0 (0 itself means "the solver's own stream" in the C ABI)
LEGACY_DEFAULT_STREAM = 1


class Solver:
    """BDDs of a 0-1 ILP on the GPU.

    ``inst`` needs attributes n, m, row_ptr, col, val, b, sense, c (CSR form; see
    ``include/bdd_dbca.h``).  ``omega`` damps the min-marginal difference; ``alpha > 0`` selects
    the smoothed (log-sum-exp) variant.  ``rank`` (a permutation of 0..n-1, or "cm" for
    :func:`cuthill_mckee`) sets the variable order of the BDD layers; ``averaging`` 1 selects
    SRMP averaging instead of eq. mma-update.  ``split`` (an interval count k >= 2) or ``cuts``
    (explicit cut places) splits the BDDs into sub-BDDs with copy-arc duals (Sec. 6), step size
    ``gamma``; ``split_depth`` D >= 1 instead cuts every BDD into pieces of at most D layers.
    ``lanes``: 1 lane tiles for BDDs of width <= 2 (one lane per BDD), 0 two-lane teams, -1
    (default) the layout tuner decides (``tune_layout``; ``layout_classes`` gives the table
    explicitly, see :meth:`layout_table`).  ``smooth_messages``: whether the smoothed forward keeps
    every sweep's messages for the gradient (1), recomputes them there (0), or keeps them when
    they fit (-1, default).
    """

    def __init__(self, inst, omega: float = 0.5, host_only: bool = False, max_device_bytes: int = 0,
                 device: int = -1, stream: int = 0, schedule: int = 1, spin_limit: int = 0,
                 alpha: float = 0.0, rank=None, averaging: int = 0, fused_pending: int = -1,
                 staging: int = -1, split: int = 0, cuts=None, gamma: float = 0.5,
                 split_depth: int = 0, lanes: int = -1, tune_layout: int = -1, layout_classes=None,
                 smooth_messages: int = -1):
        import numpy as np
        opt = B.bdd_default_options()
        if isinstance(rank, str):
            if rank != "cm":
                raise ValueError("rank must be None, 'cm' or a permutation")
            rank = cuthill_mckee(inst)
        self.rank = None if rank is None else np.ascontiguousarray(rank, np.int32)
        if self.rank is not None:
            if self.rank.shape != (inst.n,):
                raise ValueError("rank must have one entry per variable")
            opt.var_rank = self.rank.ctypes.data_as(B.C.POINTER(B.C.c_int))
        self._cuts = None if cuts is None else np.ascontiguousarray(cuts, np.int32)
        if self._cuts is not None and len(self._cuts):
            opt.cuts = self._cuts.ctypes.data_as(B.C.POINTER(B.C.c_int))
            opt.n_cuts = len(self._cuts)
        opt.split_intervals = int(split)
        opt.gamma = float(gamma)
        opt.split_depth = int(split_depth)
        opt.lanes = int(lanes)
        opt.tune_layout = int(tune_layout)
        self._layout = None if layout_classes is None else np.ascontiguousarray(layout_classes, np.int32)
        if self._layout is not None:
            if self._layout.shape != (B.BDD_LAYOUT_KEYS,):
                raise ValueError("layout_classes needs one entry per layout key")
            opt.layout_classes = self._layout.ctypes.data_as(B.C.POINTER(B.C.c_int))
        opt.averaging = int(averaging)
        opt.fused_pending = int(fused_pending)
        opt.staging = int(staging)
        opt.alpha = float(alpha)
        opt.smooth_messages = int(smooth_messages)
        opt.schedule = int(schedule)
        if spin_limit:
            opt.spin_limit = int(spin_limit)
        opt.omega = omega
        opt.host_only = int(host_only)
        opt.max_device_bytes = int(max_device_bytes)
        opt.device = int(device)
        opt.stream = stream or None
        self.h = B.bdd_build(inst.n, inst.m, inst.row_ptr, inst.col, inst.val, inst.b, inst.sense,
                             inst.c, opt)
        s = B.bdd_sizes(self.h)
        (self.n, self.m, self.nb, self.O, self.N, self.max_depth, self.max_width, self.nnz,
         self.device_bytes, self.warp_tiles, self.block_tiles, self.schedule, self.staging,
         self.n_cuts, self.npairs, self.split_depth, self.lanes, self.lane_O, self.lane_N) = map(int, s)

    def close(self):
        if getattr(self, "h", None):
            B.bdd_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def iterate(self, n_iter: int, lam: bool = False, mm: bool = False):
        """Returns (lower bound, lambda, mm0, mm1) as host arrays (None where not requested)."""
        return B.bdd_iterate(self.h, n_iter, lam=lam, mm=mm)

    def iterate_device(self, n_iter: int, trace=None, lam=None, mm0=None, mm1=None, stream=None):
        """Tensors (or raw device pointers) for the outputs; stream defaults to PyTorch's
        current stream, so the work is ordered with PyTorch's work on it."""
        def ptr(t):
            if t is None:
                return 0
            return t if isinstance(t, int) else t.data_ptr()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
            if stream == 0:
                stream = LEGACY_DEFAULT_STREAM
        B.bdd_iterate_device(self.h, n_iter, ptr(trace), ptr(lam), ptr(mm0), ptr(mm1), stream)

    def iterate_profiled(self, n_iter: int):
        """Per-kernel summed device ms: [forward sweeps, pending passes, backward sweeps,
        pending passes with bound]."""
        return B.bdd_iterate_profiled(self.h, n_iter)

    def bound_parts(self, row_off, var_off):
        """FP64 bounds of block-diagonal parts of a packed instance."""
        return B.bdd_bound_parts(self.h, row_off, var_off)

    def canonical(self) -> dict:
        return B.bdd_export_canonical(self.h)

    def get_state(self):
        return B.bdd_get_state(self.h)

    def set_state(self, lam, pending=None):
        B.bdd_set_state(self.h, lam, pending)

    def set_costs(self, c):
        B.bdd_set_costs(self.h, c)

    def layout_table(self) -> dict:
        """Tile class of every layout key and the tuner's probe times."""
        return B.bdd_layout_table(self.h)

    def cuts(self):
        """Cut places of the variable order (split solvers; empty otherwise)."""
        return B.bdd_get_cuts(self.h)

    def copy_duals(self):
        """(mu_bar, mu) of the copy-arc pairs (split solvers), canonical pair order."""
        return B.bdd_get_copy_duals(self.h)

    def set_copy_duals(self, mu_bar, mu):
        B.bdd_set_copy_duals(self.h, mu_bar, mu)


def cuthill_mckee(inst):
    """Variable order of the Cuthill-McKee search on the bipartite variable-constraint graph of
    ``inst`` (Appendix A.3); rank[i] is the place of variable i."""
    return B.bdd_cuthill_mckee(inst.n, inst.m, inst.row_ptr, inst.col, inst.val)
