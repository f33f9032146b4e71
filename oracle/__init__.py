"""FP64 oracle for BDD-based min-marginal averaging (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The product library never loads it; the two share no code.

The C source ``oracle.c`` is compiled with gcc into ``oracle/_build/liboracle.so``
(:func:`build`).  :class:`Oracle` wraps one built instance.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")

ORC_OK, ORC_EINVAL, ORC_EINFEASIBLE, ORC_ETOOBIG, ORC_ENOMEM = 0, -1, -2, -3, -4
TOP, BOT = -1, -2

_lib = None


_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle (plain C11, no FMA contraction so x86 and Arm agree bit for bit).
    omp: the OpenMP build (schedule P's loops over BDDs and variables on all host cores, the
    same results bit for bit), used only as the benchmark's second CPU baseline."""
    out = _OUT_OMP if omp else _OUT
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           *(["-fopenmp"] if omp else []), "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)
    return out


def _configure(lib):
    P = C.POINTER
    vp, i32, i64, f64 = C.c_void_p, C.c_int, C.c_longlong, C.c_double
    lib.orc_build.restype = vp
    lib.orc_build.argtypes = [i32, i32, P(i64), P(i32), P(i32), P(i32), P(C.c_byte), P(f64),
                              P(i32), P(i32)]
    lib.orc_build_ordered.restype = vp
    lib.orc_build_ordered.argtypes = [i32, i32, P(i64), P(i32), P(i32), P(i32), P(C.c_byte),
                                      P(f64), P(i32), P(i32), P(i32)]
    lib.orc_set_srmp.argtypes = [vp, i32]
    lib.orc_split.restype = i32
    lib.orc_split.argtypes = [vp, i32, P(i32), f64]
    lib.orc_split_depth.restype = i32
    lib.orc_split_depth.argtypes = [vp, i32, f64]
    lib.orc_npairs.restype = i64
    lib.orc_npairs.argtypes = [vp]
    lib.orc_get_copy_duals.argtypes = [vp, P(f64), P(f64)]
    lib.orc_set_copy_duals.argtypes = [vp, P(f64), P(f64)]
    lib.orc_free.argtypes = [vp]
    lib.orc_sizes.argtypes = [vp, P(i64)]
    lib.orc_export.argtypes = [vp, P(i32), P(i32), P(i32), P(i64), P(i32), P(i32), P(i32), P(i64)]
    lib.orc_init_dual.argtypes = [vp]
    lib.orc_worst.argtypes = [vp, P(f64)]
    lib.orc_bound.argtypes = [vp]
    lib.orc_bound.restype = f64
    lib.orc_run_parallel.argtypes = [vp, i32, f64, i32, P(f64)]
    lib.orc_run_sequential.argtypes = [vp, i32, i32, P(f64)]
    lib.orc_get_lambda.argtypes = [vp, i32, P(f64)]
    lib.orc_get_pending.argtypes = [vp, P(f64)]
    lib.orc_set_state.argtypes = [vp, P(f64), P(f64)]
    lib.orc_min_marginals.argtypes = [vp, i32, P(f64), P(f64)]
    lib.orc_energies.argtypes = [vp, P(f64)]
    lib.orc_counts.argtypes = [vp, P(f64)]
    lib.orc_set_alpha.argtypes = [vp, f64]
    lib.orc_smooth_gradient.argtypes = [vp, i32, f64, P(f64), P(f64)]
    lib.orc_smooth_gradient.restype = i32
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(C.CDLL(build()))
    return _lib


_lib_omp = None


def load_omp():
    """The OpenMP build (all host cores; see build)."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _configure(C.CDLL(build(omp=True)))
    return _lib_omp


def load_variant(path: str):
    """Load another build of oracle.c (used by the planted-mistake tests)."""
    return _configure(C.CDLL(path))


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


class OracleError(RuntimeError):
    def __init__(self, code, row):
        super().__init__(f"oracle build failed: code {code}, row {row}")
        self.code, self.row = code, row


class Oracle:
    """One instance: BDDs built from the ILP, plus FP64 dual state.

    rank: optional permutation of 0..n-1, the place of each variable in the variable order
    (Appendix A.3); BDD layers and the sequential schedule follow it.  None = identity."""

    def __init__(self, inst, lib=None, rank=None):
        lib = _load() if lib is None else lib
        self.lib = lib
        self.inst = inst
        self._keep = [np.ascontiguousarray(inst.row_ptr, np.int64),
                      np.ascontiguousarray(inst.col, np.int32),
                      np.ascontiguousarray(inst.val, np.int32),
                      np.ascontiguousarray(inst.b, np.int32),
                      np.ascontiguousarray(inst.sense, np.int8),
                      np.ascontiguousarray(inst.c, np.float64)]
        rp, col, val, b, sense, c = self._keep
        rk = None
        if rank is not None:
            rk = np.ascontiguousarray(rank, np.int32)
            if rk.shape != (inst.n,):
                raise ValueError("rank must have one entry per variable")
            self._keep.append(rk)
        st, row = C.c_int(0), C.c_int(0)
        self.h = lib.orc_build_ordered(inst.n, inst.m, _p(rp, C.c_longlong), _p(col, C.c_int),
                                       _p(val, C.c_int), _p(b, C.c_int), _p(sense, C.c_byte),
                                       _p(c, C.c_double),
                                       None if rk is None else _p(rk, C.c_int),
                                       C.byref(st), C.byref(row))
        if not self.h:
            raise OracleError(st.value, row.value)
        s = np.zeros(8, np.int64)
        lib.orc_sizes(self.h, _p(s, C.c_longlong))
        self.n, self.m, self.nb, self.O, self.N, self.max_depth, self.max_width, self.nnz = map(int, s)
        lib.orc_init_dual(self.h)

    def __del__(self):
        if getattr(self, "h", None) and getattr(self, "lib", None) is not None:
            self.lib.orc_free(self.h)
            self.h = None

    # ---- structure ---------------------------------------------------------------------
    def canonical(self) -> dict:
        """BDDs in ascending row order; occurrences BDD-major / layer-minor; nodes BDD-major,
        layer-major, canonical (ascending smallest partial sum) inside a layer."""
        bdd_row = np.zeros(self.nb, np.int32)
        bdd_depth = np.zeros(self.nb, np.int32)
        occ_var = np.zeros(self.O, np.int32)
        occ_csr = np.zeros(self.O, np.int64)
        occ_width = np.zeros(self.O, np.int32)
        lo = np.zeros(self.N, np.int32)
        hi = np.zeros(self.N, np.int32)
        minsum = np.zeros(self.N, np.int64)
        self.lib.orc_export(self.h, _p(bdd_row, C.c_int), _p(bdd_depth, C.c_int), _p(occ_var, C.c_int),
                        _p(occ_csr, C.c_longlong), _p(occ_width, C.c_int), _p(lo, C.c_int),
                        _p(hi, C.c_int), _p(minsum, C.c_longlong))
        return dict(bdd_row=bdd_row, bdd_depth=bdd_depth, occ_var=occ_var, occ_csr=occ_csr,
                    occ_width=occ_width, lo=lo, hi=hi, minsum=minsum)

    # ---- dual state --------------------------------------------------------------------
    def set_alpha(self, alpha: float):
        """Smoothing temperature (0 = min-sum); restarts the dual state."""
        self.lib.orc_set_alpha(self.h, float(alpha))

    def set_srmp(self, on: bool = True):
        """SRMP averaging (Appendix A.4) instead of eq. mma-update; restarts the dual state."""
        self.lib.orc_set_srmp(self.h, int(bool(on)))
        self.lib.orc_init_dual(self.h)

    def split(self, cuts, gamma: float = 0.5) -> int:
        """Sub-BDDs at the interval boundaries `cuts` (ascending places in the variable order;
        Sec. 6) with copy-arc step size gamma; restarts the dual state.  Returns the number of
        pieces."""
        cuts = np.ascontiguousarray(cuts, np.int32)
        self._keep.append(cuts)
        nb = self.lib.orc_split(self.h, len(cuts), _p(cuts, C.c_int) if len(cuts) else None, float(gamma))
        if nb < 0:
            raise ValueError("bad cuts or gamma")
        self.nb = nb
        self.npairs = int(self.lib.orc_npairs(self.h))
        return nb

    def split_depth(self, depth: int, gamma: float = 0.5) -> int:
        """Sub-BDDs of at most `depth` layers: every BDD of k layers is cut before layers
        floor(t k / q), t = 1 .. q-1, q = ceil(k / depth), with copy-arc step size gamma; restarts
        the dual state.  Returns the number of pieces."""
        nb = self.lib.orc_split_depth(self.h, int(depth), float(gamma))
        if nb < 0:
            raise ValueError("bad depth or gamma")
        self.nb = nb
        self.npairs = int(self.lib.orc_npairs(self.h))
        return nb

    def copy_duals(self):
        mb = np.zeros(max(self.npairs, 1))
        mu = np.zeros(max(self.npairs, 1))
        self.lib.orc_get_copy_duals(self.h, _p(mb, C.c_double), _p(mu, C.c_double))
        return mb[: self.npairs], mu[: self.npairs]

    def set_copy_duals(self, mu_bar, mu):
        mb = np.ascontiguousarray(mu_bar, np.float64)
        m = np.ascontiguousarray(mu, np.float64)
        self.lib.orc_set_copy_duals(self.h, _p(mb, C.c_double), _p(m, C.c_double))

    def reset(self):
        self.lib.orc_init_dual(self.h)

    def bound(self) -> float:
        return float(self.lib.orc_bound(self.h))

    def run_parallel(self, iters: int, omega: float = 0.5, check: bool = False) -> np.ndarray:
        tr = np.zeros(max(iters, 1), np.float64)
        self.lib.orc_run_parallel(self.h, iters, omega, int(check), _p(tr, C.c_double))
        return tr[:iters]

    def run_sequential(self, iters: int, check: bool = False) -> np.ndarray:
        tr = np.zeros(max(iters, 1), np.float64)
        rc = self.lib.orc_run_sequential(self.h, iters, int(check), _p(tr, C.c_double))
        if rc:
            raise OracleError(rc, -1)
        return tr[:iters]

    def worst(self) -> dict:
        w = np.zeros(5, np.float64)
        self.lib.orc_worst(self.h, _p(w, C.c_double))
        return dict(monotone_drop=w[0], invariant=w[1], incremental_mm=w[2], prop1=w[3],
                    negative_gain=w[4])

    def lam(self, fold: bool = True) -> np.ndarray:
        out = np.zeros(max(self.nnz, 1), np.float64)
        self.lib.orc_get_lambda(self.h, int(fold), _p(out, C.c_double))
        return out[: self.nnz]

    def pending(self) -> np.ndarray:
        out = np.zeros(max(self.n, 1), np.float64)
        self.lib.orc_get_pending(self.h, _p(out, C.c_double))
        return out[: self.n]

    def set_state(self, lam, P=None):
        lam = np.ascontiguousarray(lam, np.float64)
        if P is None:
            self.lib.orc_set_state(self.h, _p(lam, C.c_double), None)
        else:
            P = np.ascontiguousarray(P, np.float64)
            self.lib.orc_set_state(self.h, _p(lam, C.c_double), _p(P, C.c_double))

    def smooth_gradient(self, K: int, omega: float = 0.5):
        """Smoothed bound after K iterations of the deferred schedule from lambda = c/|J_i| and
        its gradient d bound / d c (FP64 reverse mode over the recorded iterations; needs
        set_alpha(alpha > 0) first).  Leaves the dual state after K iterations."""
        lb = np.zeros(1, np.float64)
        g = np.zeros(max(self.n, 1), np.float64)
        rc = self.lib.orc_smooth_gradient(self.h, int(K), float(omega), _p(lb, C.c_double), _p(g, C.c_double))
        if rc:
            raise OracleError(rc, -1)
        return float(lb[0]), g[: self.n]

    def min_marginals(self, fold: bool = True):
        m0 = np.zeros(max(self.nnz, 1), np.float64)
        m1 = np.zeros(max(self.nnz, 1), np.float64)
        self.lib.orc_min_marginals(self.h, int(fold), _p(m0, C.c_double), _p(m1, C.c_double))
        return m0[: self.nnz], m1[: self.nnz]

    def energies(self) -> np.ndarray:
        E = np.zeros(max(self.nb, 1), np.float64)
        self.lib.orc_energies(self.h, _p(E, C.c_double))
        return E[: self.nb]

    def counts(self) -> np.ndarray:
        cnt = np.zeros(max(self.nb, 1), np.float64)
        self.lib.orc_counts(self.h, _p(cnt, C.c_double))
        return cnt[: self.nb]
