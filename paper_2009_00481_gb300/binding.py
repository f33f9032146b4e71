"""ctypes binding of the C ABI (include/bdd_dbca.h).  Argument marshalling only: every step
of the method runs in the CUDA library.  There is no fallback: if the library is missing or
fails to load, loading raises.

Functions keep the C names.  Device buffers and streams may come from PyTorch: pass
``tensor.data_ptr()`` and ``torch.cuda.current_stream().cuda_stream``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, LIB_CHECKED

BDD_OK, BDD_EINVAL, BDD_EINFEASIBLE, BDD_ETOOBIG, BDD_ENOMEM = 0, -1, -2, -3, -4
BDD_ECUDA, BDD_ETIMEOUT, BDD_EDEVICE, BDD_ESTATE = -5, -6, -7, -8
BDD_SIZES_LEN = 19
BDD_LAYOUT_KEYS = 28

EXPORTED = [
    "bdd_default_options", "bdd_build", "bdd_last_failed_row", "bdd_iterate", "bdd_iterate_device",
    "bdd_iterate_profiled",
    "bdd_set_costs", "bdd_sizes", "bdd_export_canonical", "bdd_get_state", "bdd_set_state",
    "bdd_strerror", "bdd_free", "bdd_lower_bound_noalloc", "bdd_bound_parts", "bdd_smooth_forward",
    "bdd_smooth_backward", "bdd_cuthill_mckee", "bdd_get_cuts", "bdd_get_copy_duals",
    "bdd_set_copy_duals", "bdd_layout_table", "bdd_status_of_device_word",
]


class bdd_options(C.Structure):
    _fields_ = [("omega", C.c_float), ("max_width", C.c_int), ("max_nodes", C.c_longlong),
                ("max_device_bytes", C.c_longlong), ("host_only", C.c_int), ("device", C.c_int),
                ("stream", C.c_void_p), ("schedule", C.c_int), ("spin_limit", C.c_longlong),
                ("alpha", C.c_float), ("var_rank", C.POINTER(C.c_int)), ("averaging", C.c_int),
                ("fused_pending", C.c_int), ("staging", C.c_int), ("split_intervals", C.c_int),
                ("cuts", C.POINTER(C.c_int)), ("n_cuts", C.c_int), ("gamma", C.c_float),
                ("split_depth", C.c_int), ("lanes", C.c_int), ("tune_layout", C.c_int),
                ("layout_classes", C.POINTER(C.c_int)), ("smooth_messages", C.c_int)]


class BDDError(RuntimeError):
    def __init__(self, code: int, where: str, row: int = -1):
        msg = f"{where}: {strerror(code)} (status {code})"
        if row >= 0:
            msg += f", row {row}"
        super().__init__(msg)
        self.code, self.row = code, row


_lib = None


def default_library() -> str:
    """The library this process uses: the checked build (index checks in the sweep kernels
    that report BDD_EDEVICE) when the environment sets BDD_DBCA_CHECKED=1, else the normal one."""
    return LIB_CHECKED if os.environ.get("BDD_DBCA_CHECKED") == "1" else LIB


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    default = path is None
    path = path or default_library()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    P = C.POINTER
    vp, i32, i64, f32, f64 = C.c_void_p, C.c_int, C.c_longlong, C.c_float, C.c_double
    lib.bdd_default_options.argtypes = [P(bdd_options)]
    lib.bdd_default_options.restype = None
    lib.bdd_build.argtypes = [i32, i32, P(i64), P(i32), P(i32), P(i32), P(C.c_byte), P(f32),
                              P(bdd_options), P(vp)]
    lib.bdd_last_failed_row.argtypes = []
    lib.bdd_iterate.argtypes = [vp, i32, P(f64), P(f32), P(f32), P(f32)]
    lib.bdd_iterate_device.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    lib.bdd_iterate_profiled.argtypes = [vp, i32, P(f64)]
    lib.bdd_set_costs.argtypes = [vp, P(f32)]
    lib.bdd_sizes.argtypes = [vp, P(i64)]
    lib.bdd_export_canonical.argtypes = [vp, P(i32), P(i32), P(i32), P(i64), P(i32), P(i32), P(i32)]
    lib.bdd_get_state.argtypes = [vp, P(f32), P(f32)]
    lib.bdd_set_state.argtypes = [vp, P(f32), P(f32)]
    lib.bdd_strerror.argtypes = [i32]
    lib.bdd_strerror.restype = C.c_char_p
    lib.bdd_free.argtypes = [vp]
    lib.bdd_free.restype = None
    lib.bdd_lower_bound_noalloc.argtypes = [i32, i32, vp, vp, vp, f64, vp, vp]
    lib.bdd_bound_parts.argtypes = [vp, i32, P(i64), P(i64), P(f64)]
    lib.bdd_smooth_forward.argtypes = [vp, i32, vp, vp, P(i64), vp]
    lib.bdd_smooth_backward.argtypes = [vp, i64, vp, vp, vp]
    lib.bdd_cuthill_mckee.argtypes = [i32, i32, P(i64), P(i32), P(i32), P(i32)]
    lib.bdd_get_cuts.argtypes = [vp, P(i32)]
    lib.bdd_get_copy_duals.argtypes = [vp, P(f32), P(f32)]
    lib.bdd_set_copy_duals.argtypes = [vp, P(f32), P(f32)]
    lib.bdd_layout_table.argtypes = [vp, P(i64), P(i32), P(f32)]
    lib.bdd_status_of_device_word.argtypes = [i32]
    if default:
        _lib = lib
    return lib


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(C.POINTER(t))


def strerror(code: int) -> str:
    return load().bdd_strerror(int(code)).decode()


def _check(rc: int, where: str):
    if rc != BDD_OK:
        raise BDDError(rc, where)


def bdd_default_options() -> bdd_options:
    opt = bdd_options()
    load().bdd_default_options(C.byref(opt))
    return opt


def bdd_build(n, m, row_ptr, col, val, b, sense, c, opt: bdd_options | None = None) -> int:
    """Returns the solver handle (an int); raises BDDError with the failing row on error."""
    lib = load()
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.int32)
    b = np.ascontiguousarray(b, np.int32)
    sense = np.ascontiguousarray(sense, np.int8)
    c = np.ascontiguousarray(c, np.float32)
    h = C.c_void_p()
    rc = lib.bdd_build(int(n), int(m), _ptr(row_ptr, C.c_longlong), _ptr(col, C.c_int),
                       _ptr(val, C.c_int), _ptr(b, C.c_int), _ptr(sense, C.c_byte),
                       _ptr(c, C.c_float), C.byref(opt) if opt is not None else None, C.byref(h))
    if rc != BDD_OK:
        raise BDDError(rc, "bdd_build", lib.bdd_last_failed_row())
    return h.value


def bdd_cuthill_mckee(n, m, row_ptr, col, val=None) -> np.ndarray:
    """Variable order of the Cuthill-McKee search on the bipartite variable-constraint graph
    (Appendix A.3): rank[i] = place of variable i."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = None if val is None else np.ascontiguousarray(val, np.int32)
    rank = np.zeros(max(int(n), 1), np.int32)
    _check(load().bdd_cuthill_mckee(int(n), int(m), _ptr(row_ptr, C.c_longlong), _ptr(col, C.c_int),
                                    _ptr(val, C.c_int), _ptr(rank, C.c_int)), "bdd_cuthill_mckee")
    return rank[: int(n)]


def bdd_last_failed_row() -> int:
    return load().bdd_last_failed_row()


def bdd_sizes(h) -> np.ndarray:
    out = np.zeros(BDD_SIZES_LEN, np.int64)
    _check(load().bdd_sizes(h, _ptr(out, C.c_longlong)), "bdd_sizes")
    return out


def bdd_iterate(h, n_iter: int, lam: bool = False, mm: bool = False):
    """Host form: returns (lower_bound, lambda or None, mm0 or None, mm1 or None)."""
    s = bdd_sizes(h)
    nnz = int(s[7])
    lb = np.zeros(1, np.float64)
    lam_a = np.zeros(max(nnz, 1), np.float32) if lam else None
    m0 = np.zeros(max(nnz, 1), np.float32) if mm else None
    m1 = np.zeros(max(nnz, 1), np.float32) if mm else None
    _check(load().bdd_iterate(h, int(n_iter), _ptr(lb, C.c_double), _ptr(lam_a, C.c_float),
                              _ptr(m0, C.c_float), _ptr(m1, C.c_float)), "bdd_iterate")
    cut = (lambda a: None if a is None else a[:nnz])
    return float(lb[0]), cut(lam_a), cut(m0), cut(m1)


def bdd_iterate_device(h, n_iter: int, d_bound_trace=0, d_lambda=0, d_mm0=0, d_mm1=0, stream=0):
    """Device form: pointer arguments are integers (e.g. tensor.data_ptr()), 0 for none."""
    _check(load().bdd_iterate_device(h, int(n_iter), d_bound_trace or None, d_lambda or None,
                                     d_mm0 or None, d_mm1 or None, stream or None),
           "bdd_iterate_device")


def bdd_iterate_profiled(h, n_iter: int) -> np.ndarray:
    """Summed device milliseconds of [forward sweeps, pending passes, backward sweeps, pending
    passes with bound] over n_iter iterations launched kernel by kernel."""
    ms = np.zeros(4, np.float64)
    _check(load().bdd_iterate_profiled(h, int(n_iter), _ptr(ms, C.c_double)), "bdd_iterate_profiled")
    return ms


def bdd_set_costs(h, c):
    c = np.ascontiguousarray(c, np.float32)
    _check(load().bdd_set_costs(h, _ptr(c, C.c_float)), "bdd_set_costs")


def bdd_export_canonical(h) -> dict:
    s = bdd_sizes(h)
    nb, O, N = int(s[2]), int(s[3]), int(s[4])
    out = dict(bdd_row=np.zeros(max(nb, 1), np.int32), bdd_depth=np.zeros(max(nb, 1), np.int32),
               occ_var=np.zeros(max(O, 1), np.int32), occ_csr=np.zeros(max(O, 1), np.int64),
               occ_width=np.zeros(max(O, 1), np.int32), lo=np.zeros(max(N, 1), np.int32),
               hi=np.zeros(max(N, 1), np.int32))
    _check(load().bdd_export_canonical(
        h, _ptr(out["bdd_row"], C.c_int), _ptr(out["bdd_depth"], C.c_int),
        _ptr(out["occ_var"], C.c_int), _ptr(out["occ_csr"], C.c_longlong),
        _ptr(out["occ_width"], C.c_int), _ptr(out["lo"], C.c_int), _ptr(out["hi"], C.c_int)),
        "bdd_export_canonical")
    sizes = dict(bdd_row=nb, bdd_depth=nb, occ_var=O, occ_csr=O, occ_width=O, lo=N, hi=N)
    return {k: v[: sizes[k]] for k, v in out.items()}


def bdd_get_state(h):
    s = bdd_sizes(h)
    lam = np.zeros(max(int(s[7]), 1), np.float32)
    P = np.zeros(max(int(s[0]), 1), np.float32)
    _check(load().bdd_get_state(h, _ptr(lam, C.c_float), _ptr(P, C.c_float)), "bdd_get_state")
    return lam[: int(s[7])], P[: int(s[0])]


def bdd_set_state(h, lam, P=None):
    lam = np.ascontiguousarray(lam, np.float32)
    P = None if P is None else np.ascontiguousarray(P, np.float32)
    _check(load().bdd_set_state(h, _ptr(lam, C.c_float), _ptr(P, C.c_float)), "bdd_set_state")


def bdd_get_cuts(h) -> np.ndarray:
    """Cut places of a split solver (Sec. 6)."""
    k = int(bdd_sizes(h)[13])
    cuts = np.zeros(max(k, 1), np.int32)
    _check(load().bdd_get_cuts(h, _ptr(cuts, C.c_int)), "bdd_get_cuts")
    return cuts[:k]


def bdd_layout_table(h) -> dict:
    """Tile class of every layout key (natural width class c x depth bucket: key = 4 c + bucket):
    nodes, class (-1 none, 0..5 team of 2^c lanes, 6 block, 7 lane tiles) and the tuner's probe
    ms of the default and the alternative (-1: not probed)."""
    nodes = np.zeros(BDD_LAYOUT_KEYS, np.int64)
    cls = np.zeros(BDD_LAYOUT_KEYS, np.int32)
    ms = np.zeros(2 * BDD_LAYOUT_KEYS, np.float32)
    _check(load().bdd_layout_table(h, _ptr(nodes, C.c_longlong), _ptr(cls, C.c_int), _ptr(ms, C.c_float)),
           "bdd_layout_table")
    return {"nodes": nodes, "cls": cls, "ms": ms.reshape(BDD_LAYOUT_KEYS, 2)}


def bdd_get_copy_duals(h):
    """(mu_bar, mu) of every copy-arc pair, canonical pair order."""
    k = int(bdd_sizes(h)[14])
    mb = np.zeros(max(k, 1), np.float32)
    mu = np.zeros(max(k, 1), np.float32)
    _check(load().bdd_get_copy_duals(h, _ptr(mb, C.c_float), _ptr(mu, C.c_float)), "bdd_get_copy_duals")
    return mb[:k], mu[:k]


def bdd_set_copy_duals(h, mu_bar, mu):
    mb = np.ascontiguousarray(mu_bar, np.float32)
    m = np.ascontiguousarray(mu, np.float32)
    _check(load().bdd_set_copy_duals(h, _ptr(mb, C.c_float), _ptr(m, C.c_float)), "bdd_set_copy_duals")


def bdd_lower_bound_noalloc(n: int, nb: int, d_E: int, d_P: int, d_deg: int, empty_const: float,
                            d_bound: int, stream: int = 0):
    """Bound reduction into caller device memory with no allocation (pointers are integers,
    e.g. tensor.data_ptr()).  For callers that cannot allocate device memory."""
    _check(load().bdd_lower_bound_noalloc(int(n), int(nb), d_E or None, d_P or None, d_deg or None,
                                          float(empty_const), d_bound or None, stream or None),
           "bdd_lower_bound_noalloc")


def bdd_bound_parts(h, row_off, var_off) -> np.ndarray:
    """FP64 bounds of block-diagonal parts (row / variable offsets, each nparts + 1 long)."""
    row_off = np.ascontiguousarray(row_off, np.int64)
    var_off = np.ascontiguousarray(var_off, np.int64)
    out = np.zeros(len(row_off) - 1, np.float64)
    _check(load().bdd_bound_parts(h, len(out), _ptr(row_off, C.c_longlong), _ptr(var_off, C.c_longlong),
                                  _ptr(out, C.c_double)), "bdd_bound_parts")
    return out


def bdd_smooth_forward(h, K: int, d_c: int, d_bound: int, stream: int = 0) -> int:
    """Smoothed bound after K iterations from costs c (device pointers as integers).  Returns
    the forward's generation number, which bdd_smooth_backward needs."""
    gen = C.c_longlong(-1)
    _check(load().bdd_smooth_forward(h, int(K), d_c or None, d_bound or None, C.byref(gen), stream or None),
           "bdd_smooth_forward")
    return int(gen.value)


def bdd_smooth_backward(h, generation: int, d_gbound: int, d_grad_c: int, stream: int = 0):
    """g * d(smoothed bound)/dc into d_grad_c for the forward that returned `generation`
    (BDDError with BDD_ESTATE if it is no longer the solver's last forward)."""
    _check(load().bdd_smooth_backward(h, int(generation), d_gbound or None, d_grad_c or None, stream or None),
           "bdd_smooth_backward")


def bdd_strerror(code: int) -> str:
    return strerror(code)


def bdd_free(h):
    if h:
        load().bdd_free(h)
