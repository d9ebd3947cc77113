"""ctypes front end of the C oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sogrand_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, IEEE FP64, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Code(C.Structure):
    _fields_ = [("n", C.c_int), ("k", C.c_int), ("H", C.POINTER(C.c_uint8)), ("even", C.c_int),
                ("reading", C.c_int), ("c_max", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = np.ctypeslib.ndpointer
            L.oracle_one_line_c.argtypes = [C.c_int, P(np.float32, flags="C"), C.c_int]
            L.oracle_one_line_c.restype = C.c_int
            L.oracle_trace.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
            L.oracle_trace.restype = C.c_int64
            L.oracle_siso.argtypes = [C.POINTER(_Code), C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_double,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.oracle_siso.restype = C.c_int
            L.oracle_product.argtypes = [C.POINTER(_Code), C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_float,
                                         C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.oracle_product.restype = C.c_int
            L.oracle_product2.argtypes = [C.POINTER(_Code), C.POINTER(_Code), C.c_void_p, C.c_int, C.c_int64,
                                          C.c_double, C.c_float, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]
            L.oracle_product2.restype = C.c_int
            L.oracle_product_trace.argtypes = L.oracle_product2.argtypes + [C.c_void_p]
            L.oracle_product_trace.restype = C.c_int
            L.oracle_gldpc.argtypes = L.oracle_product.argtypes
            L.oracle_gldpc.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleCode:
    """Oracle view of a linear code: H plus the even/reading/c_max options.

    reading 0: the parity-class normalisation (reading B); 1: the literal one
    (reading A); 2: Forney's approximation, APPs normalised over the list.
    """

    def __init__(self, code, even: bool | None = None, reading: int = 0, c_max: int | None = None):
        self.code = code
        self.n, self.k = code.n, code.k
        self.H = np.ascontiguousarray(code.H, dtype=np.uint8)
        self.even = bool(code.even if even is None else even)
        self.reading = int(reading)
        self.c_max = int(code.n if c_max is None else c_max)
        self._s = _Code(self.n, self.k, self.H.ctypes.data_as(C.POINTER(C.c_uint8)), int(self.even),
                        self.reading, self.c_max)


def one_line_c(absl_sorted, c_max: int) -> int:
    a = np.ascontiguousarray(absl_sorted, dtype=np.float32)
    return int(lib().oracle_one_line_c(a.size, a, int(c_max)))


def trace(n: int, c: int, cls: int, max_q: int):
    """Canonical 1-line ORBGRAND order: (rank masks [q, n] u8, cost [q], weight [q])."""
    ranks = np.zeros((max_q, n), dtype=np.uint8)
    cost = np.zeros(max_q, dtype=np.int32)
    w = np.zeros(max_q, dtype=np.int32)
    q = lib().oracle_trace(n, c, cls, max_q, _ptr(ranks), _ptr(cost), _ptr(w))
    return ranks[:q], cost[:q], w[:q]


def siso(oc: OracleCode, lch, la=None, L: int = 4, cap: int = 10**4, thr: float = 0.0) -> dict:
    n = oc.n
    lch = np.ascontiguousarray(lch, dtype=np.float32)
    la = None if la is None else np.ascontiguousarray(la, dtype=np.float32)
    out = dict(lapp=np.zeros(n), lext=np.zeros(n), hard=np.zeros(n, np.uint8), pmiss=np.zeros(1),
               queries=np.zeros(1, np.int64), list_count=np.zeros(1, np.int32),
               list_words=np.zeros((L, n), np.uint8), list_logp=np.zeros(L), list_app=np.zeros(L),
               list_q=np.zeros(L, np.int64), diag=np.zeros(10))
    rc = lib().oracle_siso(C.byref(oc._s), _ptr(lch), _ptr(la), L, cap, thr, _ptr(out["lapp"]), _ptr(out["lext"]),
                           _ptr(out["hard"]), _ptr(out["pmiss"]), _ptr(out["queries"]), _ptr(out["list_count"]),
                           _ptr(out["list_words"]), _ptr(out["list_logp"]), _ptr(out["list_app"]),
                           _ptr(out["list_q"]), _ptr(out["diag"]))
    if rc == -2:
        raise ValueError("invalid oracle arguments")
    out["rc"] = rc
    out["pmiss"] = float(out["pmiss"][0])
    out["queries"] = int(out["queries"][0])
    nl = int(out["list_count"][0])
    out["list_count"] = nl
    for key in ("list_words", "list_logp", "list_app", "list_q"):
        out[key] = out[key][:nl]
    d = out["diag"]
    out.update(c=int(d[0]), cstar=int(d[1]), level_idx=int(d[2]), log_r=d[3], log_r_direct=d[4], S=d[5],
               log_phi=d[6], exhausted=bool(d[7]), parity=int(d[8]), thr_stop=bool(d[9]))
    return out


def _threads(threads):
    return threads or os.cpu_count() or 1


def siso_batch(oc: OracleCode, lch, la=None, L=4, cap=10**4, thr=0.0, threads=None) -> dict:
    """Many words ([W, n]) on all host cores; returns stacked arrays."""
    lch = np.ascontiguousarray(lch, dtype=np.float32)
    W = lch.shape[0]
    res = [None] * W

    def one(i):
        res[i] = siso(oc, lch[i], None if la is None else la[i], L, cap, thr)

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(W)))
    return dict(lapp=np.stack([r["lapp"] for r in res]), lext=np.stack([r["lext"] for r in res]),
                hard=np.stack([r["hard"] for r in res]), pmiss=np.array([r["pmiss"] for r in res]),
                queries=np.array([r["queries"] for r in res], np.int64),
                list_count=np.array([r["list_count"] for r in res], np.int32), items=res)


def product(oc: OracleCode, lch, L=4, cap=10**4, thr=0.0, alpha=0.5, max_iter=20, col: OracleCode | None = None) -> dict:
    """One frame (row-major [n_col, n_row]) of the product of the row code `oc`
    and the column code `col` (default: `oc`, a square product code)."""
    col = oc if col is None else col
    nr, nc = oc.n, col.n
    lch = np.ascontiguousarray(lch, dtype=np.float32).reshape(nr * nc)
    bits = np.zeros(nr * nc, np.uint8)
    hi = np.zeros(1, np.int32)
    st = np.zeros(1, np.uint8)
    q = np.zeros(1, np.int64)
    qp = np.zeros(1, np.int64)
    lib().oracle_product2(C.byref(oc._s), C.byref(col._s), _ptr(lch), L, cap, thr, C.c_float(alpha), max_iter,
                          _ptr(bits), _ptr(hi), _ptr(st), _ptr(q), _ptr(qp))
    return dict(bits=bits.reshape(nc, nr), half_iters=int(hi[0]), status=int(st[0]), queries=int(q[0]),
                par_queries=int(qp[0]))


def product_trace(oc: OracleCode, lch, L=4, cap=10**4, thr=0.0, alpha=0.5, max_iter=20,
                  col: OracleCode | None = None) -> dict:
    """product() of one frame with the L_APP of every half iteration:
    lapp_trace [2 max_iter, n_col, n_row] (NaN for halves not run)."""
    col = oc if col is None else col
    nr, nc = oc.n, col.n
    lch = np.ascontiguousarray(lch, dtype=np.float32).reshape(nr * nc)
    bits = np.zeros(nr * nc, np.uint8)
    hi = np.zeros(1, np.int32)
    st = np.zeros(1, np.uint8)
    q = np.zeros(1, np.int64)
    qp = np.zeros(1, np.int64)
    tr = np.full((2 * max_iter, nc, nr), np.nan)
    lib().oracle_product_trace(C.byref(oc._s), C.byref(col._s), _ptr(lch), L, cap, thr, C.c_float(alpha), max_iter,
                               _ptr(bits), _ptr(hi), _ptr(st), _ptr(q), _ptr(qp), _ptr(tr))
    return dict(bits=bits.reshape(nc, nr), half_iters=int(hi[0]), status=int(st[0]), queries=int(q[0]),
                par_queries=int(qp[0]), lapp_trace=tr)


def gldpc(oc: OracleCode, lch, L=4, cap=10**4, thr=0.0, alpha=0.5, max_iter=20) -> dict:
    """One frame [n, n] of the QC-GLDPC code of component `oc` (rows and wrapped diagonals)."""
    n = oc.n
    lch = np.ascontiguousarray(lch, dtype=np.float32).reshape(n * n)
    bits = np.zeros(n * n, np.uint8)
    hi = np.zeros(1, np.int32)
    st = np.zeros(1, np.uint8)
    q = np.zeros(1, np.int64)
    qp = np.zeros(1, np.int64)
    lib().oracle_gldpc(C.byref(oc._s), _ptr(lch), L, cap, thr, C.c_float(alpha), max_iter, _ptr(bits), _ptr(hi),
                       _ptr(st), _ptr(q), _ptr(qp))
    return dict(bits=bits.reshape(n, n), half_iters=int(hi[0]), status=int(st[0]), queries=int(q[0]),
                par_queries=int(qp[0]))


def gldpc_batch(oc: OracleCode, lch, L=4, cap=10**4, thr=0.0, alpha=0.5, max_iter=20, threads=None) -> dict:
    lch = np.ascontiguousarray(lch, dtype=np.float32)
    F = lch.shape[0]
    res = [None] * F

    def one(i):
        res[i] = gldpc(oc, lch[i], L, cap, thr, alpha, max_iter)

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(F)))
    return dict(bits=np.stack([r["bits"] for r in res]), half_iters=np.array([r["half_iters"] for r in res]),
                status=np.array([r["status"] for r in res]), queries=np.array([r["queries"] for r in res]),
                par_queries=np.array([r["par_queries"] for r in res]))


def product_batch(oc: OracleCode, lch, L=4, cap=10**4, thr=0.0, alpha=0.5, max_iter=20, threads=None,
                  col: OracleCode | None = None) -> dict:
    lch = np.ascontiguousarray(lch, dtype=np.float32)
    F = lch.shape[0]
    res = [None] * F

    def one(i):
        res[i] = product(oc, lch[i], L, cap, thr, alpha, max_iter, col)

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(F)))
    return dict(bits=np.stack([r["bits"] for r in res]), half_iters=np.array([r["half_iters"] for r in res]),
                status=np.array([r["status"] for r in res]), queries=np.array([r["queries"] for r in res]),
                par_queries=np.array([r["par_queries"] for r in res]))
