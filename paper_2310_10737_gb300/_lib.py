"""ctypes binding of libsogrand (include/sogrand.h).  Argument marshalling only:
every step of decoding runs in the library's CUDA kernels.  PyTorch supplies
device memory and the current stream.

The library must have been built (``python -m paper_2310_10737_gb300.build`` or
``__graft_entry__.build()``); importing the decode functions without it raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsogrand.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)

_lock = threading.Lock()
_lib = None


class ProductStats(C.Structure):
    """product_decode_stats of include/sogrand.h."""
    _fields_ = [("par_queries", C.c_void_p), ("weight_sum", C.c_void_p), ("xf_words", C.c_void_p),
                ("timing_ms", C.POINTER(C.c_float)), ("launches", C.POINTER(C.c_int32)),
                ("le_trace", C.c_void_p), ("word_queries", C.c_void_p)]


class SograndError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class FrameGroup(C.Structure):
    """sogrand_frame_group: one code's frames in a mixed launch."""
    _fields_ = [("code", C.c_void_p), ("n_frames", C.c_int64), ("llr_ch", C.c_void_p), ("bits", C.c_void_p),
                ("half_iters", C.c_void_p), ("status", C.c_void_p), ("queries", C.c_void_p)]


def load() -> C.CDLL:
    """Load libsogrand.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2310_10737_gb300.build` "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, f32 = C.c_void_p, C.c_int64, C.c_int, C.c_float
        L.sogrand_code_create.argtypes = [i32, i32, vp, i32, C.POINTER(vp)]
        L.sogrand_code_destroy.argtypes = [vp]
        L.sogrand_code_destroy.restype = None
        L.sogrand_code_reserve.argtypes = [vp, i64]
        L.sogrand_code_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.sogrand_set_wait_limits.argtypes = [i64, i64, i32]
        L.sogrand_code_tables.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.sogrand_decode.argtypes = [vp, i64, vp, vp, i32, i64, f32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.sogrand_decode_forney.argtypes = [vp, i64, vp, vp, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.product_decode.argtypes = [vp, vp, i64, vp, i32, i64, f32, f32, i32, vp, vp, vp, vp, vp]
        L.product_decode_ex.argtypes = [vp, vp, i64, vp, i32, i64, f32, f32, i32, vp, vp, vp, vp,
                                        C.POINTER(ProductStats), vp]
        L.product_decode_host.argtypes = [vp, vp, i64, vp, i32, i64, f32, f32, i32, vp, vp, vp, vp, vp]
        L.product_decode_persistent.argtypes = [vp, vp, i64, vp, i32, i64, f32, f32, i32, vp, vp, vp, vp,
                                                C.POINTER(ProductStats), vp]
        L.sogrand_trace_patterns.argtypes = [vp, vp, i64, vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
        L.sogrand_release_cached.argtypes = []
        L.gldpc_decode.argtypes = [vp, i64, vp, i32, i64, f32, f32, i32, vp, vp, vp, vp, C.POINTER(ProductStats), vp]
        L.sogrand_server_create.argtypes = [i32, C.POINTER(vp), C.POINTER(C.c_int64), i32, i64, f32, f32, i32, i32,
                                            C.POINTER(vp)]
        L.sogrand_server_submit.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, C.POINTER(C.c_int64)]
        L.sogrand_server_wait.argtypes = [vp, i64, i32, C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.sogrand_server_stats.argtypes = [vp] + [C.POINTER(C.c_int64)] * 5
        L.sogrand_server_destroy.argtypes = [vp]
        L.sogrand_code_schedule.argtypes = [vp, i32, C.POINTER(C.c_int)]
        L.sogrand_code_dp_area.argtypes = [vp, i32, C.POINTER(C.c_int)]
        L.sogrand_code_order_source.argtypes = [vp, i32, C.POINTER(C.c_int)]
        L.sogrand_code_tune.argtypes = [vp, i64, vp, i32, i64, f32, f32, i32, C.POINTER(C.c_int),
                                        C.POINTER(C.c_float), vp]
        L.product_decode_mixed.argtypes = [i32, C.POINTER(FrameGroup), i32, i64, f32, f32, i32,
                                           C.POINTER(ProductStats), vp]
        L.sogrand_int_peak.argtypes = [i64, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        L.sogrand_strerror.argtypes = [i32]
        L.sogrand_strerror.restype = C.c_char_p
        for name in ("sogrand_code_create", "sogrand_code_reserve", "sogrand_code_info", "sogrand_set_wait_limits",
                     "sogrand_code_tables", "sogrand_decode",
                     "sogrand_decode_forney",
                     "product_decode", "product_decode_ex", "product_decode_host", "product_decode_persistent",
                     "sogrand_trace_patterns", "sogrand_release_cached", "sogrand_int_peak",
                     "product_decode_mixed", "sogrand_code_schedule", "sogrand_code_dp_area", "sogrand_code_order_source", "sogrand_code_tune", "sogrand_server_create",
                     "gldpc_decode",
                     "sogrand_server_submit", "sogrand_server_wait", "sogrand_server_stats", "sogrand_server_destroy"):
            getattr(L, name).restype = C.c_int
        _lib = L
        return L


def strerror(code: int) -> str:
    try:
        return load().sogrand_strerror(code).decode()
    except RuntimeError:
        return f"error {code}"


def _check(rc: int, where: str):
    if rc != OK:
        raise SograndError(rc, where)


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Code:
    """A component code on the current device (sogrand_code_create)."""

    def __init__(self, H, even: bool = True):
        H = np.ascontiguousarray(H, dtype=np.uint8)
        m, n = H.shape
        self.n, self.k, self.m = n, n - m, m
        self._H = H
        h = C.c_void_p()
        _check(load().sogrand_code_create(n, n - m, H.ctypes.data_as(C.c_void_p), int(bool(even)), C.byref(h)),
               "sogrand_code_create")
        self._h = h

    @classmethod
    def from_linear_code(cls, code, even=None):
        return cls(code.H, code.even if even is None else even)

    @property
    def handle(self):
        return self._h

    def reserve(self, max_query_cap: int):
        _check(load().sogrand_code_reserve(self._h, int(max_query_cap)), "sogrand_code_reserve")

    def tables(self):
        """(query cap the order tables cover, their device bytes)."""
        cap, nb = C.c_int64(0), C.c_int64(0)
        _check(load().sogrand_code_tables(self._h, C.byref(cap), C.byref(nb)), "sogrand_code_tables")
        return cap.value, nb.value

    def schedule(self, minb: int = 0) -> int:
        """Set (8 or 12) or query (0) the blocks per SM the decoding kernels run at."""
        cur = C.c_int(0)
        _check(load().sogrand_code_schedule(self.handle, int(minb), C.byref(cur)), "sogrand_code_schedule")
        return cur.value

    def dp_area(self, where: int = -1) -> int:
        """Set (0 shared, 1 global) or query (-1) where the batched forms keep the remaining-mass area."""
        cur = C.c_int(0)
        _check(load().sogrand_code_dp_area(self.handle, int(where), C.byref(cur)), "sogrand_code_dp_area")
        return cur.value

    def order_source(self, source: int = -1) -> int:
        """Set (0 order table, 1 lanes enumerate the order) or query (-1) where the query loop takes its patterns."""
        cur = C.c_int(0)
        _check(load().sogrand_code_order_source(self.handle, int(source), C.byref(cur)), "sogrand_code_order_source")
        return cur.value

    def tune(self, llr_sample, L: int = 4, query_cap: int = 10**4, thr: float = 0.0, alpha: float = 0.5,
             max_iter: int = 20, stream=None):
        """Autotune the schedule on a device sample [F, n, n]; returns (chosen, (ms at 8, ms at 12))."""
        ch = C.c_int(0)
        ms = (C.c_float * 2)()
        _check(load().sogrand_code_tune(self.handle, int(llr_sample.shape[0]), _ptr(llr_sample), int(L),
                                        int(query_cap), float(thr), float(alpha), int(max_iter), C.byref(ch),
                                        C.cast(ms, C.POINTER(C.c_float)), _stream(stream)), "sogrand_code_tune")
        return ch.value, (float(ms[0]), float(ms[1]))

    def close(self):
        if getattr(self, "_h", None):
            load().sogrand_code_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sogrand_code_create(H, even: bool = True) -> Code:
    return Code(H, even)


def sogrand_decode(code: Code, llr_ch, llr_a=None, L: int = 4, query_cap: int = 10**4, thr: float = 0.0,
                   lists: bool = True, stream=None, forney: bool = False) -> dict:
    """Decode the rows of ``llr_ch`` ([W, n] float32 CUDA tensor); returns CUDA tensors.
    forney=True: Forney's list-only normalisation (sogrand_decode_forney)."""
    import torch
    W, n = llr_ch.shape
    assert n == code.n and llr_ch.is_cuda and llr_ch.dtype == torch.float32 and llr_ch.is_contiguous()
    if llr_a is not None:
        assert llr_a.shape == llr_ch.shape and llr_a.dtype == torch.float32 and llr_a.is_contiguous()
    dev = llr_ch.device
    nm = (n + 63) // 64
    out = dict(hard=torch.empty((W, n), dtype=torch.uint8, device=dev),
               llr_app=torch.empty((W, n), dtype=torch.float32, device=dev),
               llr_ext=torch.empty((W, n), dtype=torch.float32, device=dev),
               p_miss=torch.empty(W, dtype=torch.float32, device=dev),
               queries=torch.empty(W, dtype=torch.int64, device=dev))
    if lists:
        out.update(list_words=torch.empty((W, L, nm), dtype=torch.int64, device=dev),
                   list_app=torch.empty((W, L), dtype=torch.float32, device=dev),
                   list_count=torch.empty(W, dtype=torch.int32, device=dev))
    tail = (_ptr(out["hard"]), _ptr(out["llr_app"]), _ptr(out["llr_ext"]), _ptr(out["p_miss"]), _ptr(out["queries"]),
            _ptr(out.get("list_words")), _ptr(out.get("list_app")), _ptr(out.get("list_count")), _stream(stream))
    if forney:
        assert thr == 0.0, "Forney's normalisation has no threshold rule"
        rc = load().sogrand_decode_forney(code.handle, W, _ptr(llr_ch), _ptr(llr_a), int(L), int(query_cap), *tail)
    else:
        rc = load().sogrand_decode(code.handle, W, _ptr(llr_ch), _ptr(llr_a), int(L), int(query_cap), float(thr),
                                   *tail)
    _check(rc, "sogrand_decode_forney" if forney else "sogrand_decode")
    return out


def product_decode(code: Code, llr_ch, L: int = 4, query_cap: int = 10**4, thr: float = 0.0, alpha: float = 0.5,
                   max_iter: int = 20, col_code: Code | None = None, stream=None, out=None, stats: bool = True,
                   persistent: bool = False, trace: bool = False) -> dict:
    """Decode [F, n, n] frames (float32 CUDA tensor); returns CUDA tensors (and,
    with stats, host-side timing_ms / launches).  persistent=True uses the
    batched form (product_decode_persistent), else one launch per half
    (product_decode_ex).  trace=True (plain form) also returns le_trace
    [2 max_iter, F, n_col, n_row] (L_E after every half) and word_queries
    [2 max_iter, F, max(n_row, n_col)] (queries of every word of every half)."""
    import torch
    cc = col_code if col_code is not None else code
    F, nc, nr = llr_ch.shape  # frames of n_col rows (column code's n) by n_row columns (row code's n)
    assert nr == code.n and nc == cc.n and llr_ch.is_cuda and llr_ch.dtype == torch.float32 and llr_ch.is_contiguous()
    dev = llr_ch.device
    if out is None:
        out = dict(bits=torch.empty((F, (nr * nc + 7) // 8), dtype=torch.uint8, device=dev),
                   half_iters=torch.empty(F, dtype=torch.int32, device=dev),
                   status=torch.empty(F, dtype=torch.uint8, device=dev),
                   queries=torch.empty(F, dtype=torch.int64, device=dev),
                   par_queries=torch.empty(F, dtype=torch.int64, device=dev),
                   weight_sum=torch.zeros(1, dtype=torch.int64, device=dev),
                   xf_words=torch.zeros(1, dtype=torch.int32, device=dev))
    st = None
    if trace:
        assert not persistent, "per-half traces come from the plain form"
        stats = True
        out["le_trace"] = torch.full((2 * max_iter, F, nc, nr), float("nan"), dtype=torch.float32, device=dev)
        out["word_queries"] = torch.full((2 * max_iter, F, max(nr, nc)), -2, dtype=torch.int32, device=dev)
    if stats:
        tm = (C.c_float * 2)()
        ln = (C.c_int32 * 1)()
        st = ProductStats(_ptr(out.get("par_queries")), _ptr(out.get("weight_sum")), _ptr(out.get("xf_words")),
                          C.cast(tm, C.POINTER(C.c_float)), C.cast(ln, C.POINTER(C.c_int32)),
                          _ptr(out.get("le_trace")), _ptr(out.get("word_queries")))
    fn = load().product_decode_persistent if persistent else load().product_decode_ex
    rc = fn(code.handle, cc.handle, F, _ptr(llr_ch), int(L), int(query_cap), float(thr), float(alpha), int(max_iter),
            _ptr(out["bits"]), _ptr(out.get("half_iters")), _ptr(out.get("status")), _ptr(out.get("queries")),
            C.byref(st) if st is not None else None, _stream(stream))
    _check(rc, "product_decode_persistent" if persistent else "product_decode")
    if stats:
        out["timing_ms"] = (float(tm[0]), float(tm[1]))
        out["launches"] = int(ln[0])
    return out


def gldpc_decode(code: Code, llr_ch, L: int = 4, query_cap: int = 10**4, thr: float = 0.0, alpha: float = 0.6,
                 max_iter: int = 20, stream=None) -> dict:
    """QC-GLDPC frames [F, n, n] (rows and wrapped diagonals are component words); returns CUDA tensors."""
    import torch
    F, n, n2 = llr_ch.shape
    assert n == n2 == code.n and llr_ch.is_cuda and llr_ch.dtype == torch.float32 and llr_ch.is_contiguous()
    dev = llr_ch.device
    out = dict(bits=torch.empty((F, (n * n + 7) // 8), dtype=torch.uint8, device=dev),
               half_iters=torch.empty(F, dtype=torch.int32, device=dev),
               status=torch.empty(F, dtype=torch.uint8, device=dev),
               queries=torch.empty(F, dtype=torch.int64, device=dev),
               par_queries=torch.empty(F, dtype=torch.int64, device=dev))
    tm = (C.c_float * 2)()
    st = ProductStats(_ptr(out["par_queries"]), None, None, C.cast(tm, C.POINTER(C.c_float)), None)
    rc = load().gldpc_decode(code.handle, F, _ptr(llr_ch), int(L), int(query_cap), float(thr), float(alpha),
                             int(max_iter), _ptr(out["bits"]), _ptr(out["half_iters"]), _ptr(out["status"]),
                             _ptr(out["queries"]), C.byref(st), _stream(stream))
    _check(rc, "gldpc_decode")
    out["timing_ms"] = float(tm[0])
    return out


def product_decode_mixed(groups, L: int = 4, query_cap: int = 10**4, thr: float = 0.0, alpha: float = 0.5,
                         max_iter: int = 20, stream=None, stats: bool = True):
    """Frames of several codes in one launch.  groups: list of (Code, llr [F, n, n] float32 CUDA tensor).
    Returns (list of per-group output dicts of CUDA tensors, info dict)."""
    import torch
    outs, arr = [], (FrameGroup * len(groups))()
    for g, (code, llr) in enumerate(groups):
        F, n, n2 = llr.shape
        assert n == n2 == code.n and llr.is_cuda and llr.dtype == torch.float32 and llr.is_contiguous()
        dev = llr.device
        o = dict(bits=torch.empty((F, (n * n + 7) // 8), dtype=torch.uint8, device=dev),
                 half_iters=torch.empty(F, dtype=torch.int32, device=dev),
                 status=torch.empty(F, dtype=torch.uint8, device=dev),
                 queries=torch.empty(F, dtype=torch.int64, device=dev))
        outs.append(o)
        arr[g] = FrameGroup(code.handle, F, _ptr(llr), _ptr(o["bits"]), _ptr(o["half_iters"]), _ptr(o["status"]),
                            _ptr(o["queries"]))
    info = {}
    st = None
    if stats:
        dev = groups[0][1].device
        info["weight_sum"] = torch.zeros(1, dtype=torch.int64, device=dev)
        info["xf_words"] = torch.zeros(1, dtype=torch.int32, device=dev)
        tm = (C.c_float * 2)()
        ln = (C.c_int32 * 1)()
        st = ProductStats(None, _ptr(info["weight_sum"]), _ptr(info["xf_words"]), C.cast(tm, C.POINTER(C.c_float)),
                          C.cast(ln, C.POINTER(C.c_int32)))
    rc = load().product_decode_mixed(len(groups), arr, int(L), int(query_cap), float(thr), float(alpha), int(max_iter),
                                     C.byref(st) if st is not None else None, _stream(stream))
    _check(rc, "product_decode_mixed")
    if stats:
        info["timing_ms"] = float(tm[0])
        info["launches"] = int(ln[0])
    return outs, info


def product_decode_host(code: Code, llr_ch: np.ndarray, L: int = 4, query_cap: int = 10**4, thr: float = 0.0,
                        alpha: float = 0.5, max_iter: int = 20, out=None, stream=None,
                        col_code: Code | None = None) -> dict:
    """product_decode on HOST buffers (numpy or pinned CPU torch tensors); copies inside the call."""
    cc = col_code if col_code is not None else code
    F, nc, nr = llr_ch.shape
    assert nr == code.n and nc == cc.n
    if out is None:
        out = dict(bits=np.empty((F, (nr * nc + 7) // 8), np.uint8), half_iters=np.empty(F, np.int32),
                   status=np.empty(F, np.uint8), queries=np.empty(F, np.int64))

    def hp(a):
        if a is None:
            return None
        return C.c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else a.ctypes.data_as(C.c_void_p)

    rc = load().product_decode_host(code.handle, cc.handle, F, hp(llr_ch), int(L), int(query_cap), float(thr),
                                    float(alpha), int(max_iter), hp(out["bits"]), hp(out["half_iters"]),
                                    hp(out["status"]), hp(out["queries"]), _stream(stream))
    _check(rc, "product_decode_host")
    return out


class Server:
    """Continuous-batching decode server (sogrand_server_*): requests of
    registered codes are admitted into device-resident frame slots as they
    free up and decoded in epochs of half iterations."""

    def __init__(self, codes, slots, L: int = 4, query_cap: int = 10**4, thr: float = 0.0, alpha: float = 0.5,
                 max_iter: int = 20, epoch_halves: int = 2):
        self.codes = list(codes)
        hs = (C.c_void_p * len(self.codes))(*[c.handle for c in self.codes])
        sl = (C.c_int64 * len(self.codes))(*[int(x) for x in slots])
        h = C.c_void_p()
        _check(load().sogrand_server_create(len(self.codes), hs, sl, int(L), int(query_cap), float(thr), float(alpha),
                                            int(max_iter), int(epoch_halves), C.byref(h)), "sogrand_server_create")
        self._h = h
        self._keep = {}

    def submit(self, code_index: int, llr, out=None):
        """Queue host frames [F, n, n] float32 (numpy or pinned torch); returns (ticket, out dict of host arrays)."""
        code = self.codes[code_index]
        F, n, _ = llr.shape
        assert n == code.n
        if out is None:
            out = dict(bits=np.empty((F, (n * n + 7) // 8), np.uint8), half_iters=np.empty(F, np.int32),
                       status=np.empty(F, np.uint8), queries=np.empty(F, np.int64))

        def hp(a):
            return C.c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else a.ctypes.data_as(C.c_void_p)

        t = C.c_int64(0)
        _check(load().sogrand_server_submit(self._h, int(code_index), int(F), hp(llr), hp(out["bits"]),
                                            hp(out["half_iters"]), hp(out["status"]), hp(out["queries"]),
                                            C.byref(t)), "sogrand_server_submit")
        self._keep[t.value] = (llr, out)
        return t.value, out

    def wait(self, ticket: int, timeout_ms: int = 60000):
        """(done, latency_ms); raises SograndError if the request failed."""
        done, lat = C.c_int(0), C.c_double(0)
        rc = load().sogrand_server_wait(self._h, int(ticket), int(timeout_ms), C.byref(done), C.byref(lat))
        if done.value:
            self._keep.pop(ticket, None)
        _check(rc, "sogrand_server_wait")
        return bool(done.value), lat.value

    def stats(self):
        v = [C.c_int64(0) for _ in range(5)]
        load().sogrand_server_stats(self._h, *[C.byref(x) for x in v])
        return dict(zip(("launches", "frames_done", "requests_done", "frames_resident", "requests_waiting"),
                        [x.value for x in v]))

    def close(self):
        if getattr(self, "_h", None):
            rc = load().sogrand_server_destroy(self._h)
            self._h = None
            self._keep.clear()
            _check(rc, "sogrand_server_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sogrand_set_wait_limits(queue_wait_us: int = -1, lock_polls: int = -1, lock_preheld: int = -1):
    """Limits of the bounded device waits (negative: keep); see include/sogrand.h."""
    _check(load().sogrand_set_wait_limits(int(queue_wait_us), int(lock_polls), int(lock_preheld)),
           "sogrand_set_wait_limits")


DEFAULT_QUEUE_WAIT_US, DEFAULT_LOCK_POLLS = 2_000_000, 1 << 22


def sogrand_release_cached():
    """Return the idle memory of the library's device pools (call after synchronising)."""
    _check(load().sogrand_release_cached(), "sogrand_release_cached")


def sogrand_int_peak(trips: int = 150_000, stream=None):
    """Measured integer-pipe rate of the current device: (lane-ops/s, kernel ms)."""
    ops, ms = C.c_double(0), C.c_double(0)
    _check(load().sogrand_int_peak(int(trips), C.byref(ops), C.byref(ms), _stream(stream)), "sogrand_int_peak")
    return ops.value, ms.value


def unpack_bits(bits, n: int, n_row: int | None = None):
    """[F, ceil(n*n_row/8)] u8 (LSB first) -> [F, n, n_row] u8 (numpy); n_row defaults to n."""
    nr = n if n_row is None else n_row
    b = np.asarray(bits.cpu() if hasattr(bits, "cpu") else bits, dtype=np.uint8)
    F = b.shape[0]
    return np.unpackbits(b, axis=1, bitorder="little")[:, :n * nr].reshape(F, n, nr)


def unpack_words(words, n: int):
    """[..., ceil(n/64)] int64 bit masks -> [..., n] u8 (numpy)."""
    w = np.asarray(words.cpu() if hasattr(words, "cpu") else words).view(np.uint64)
    bytes_ = w.astype("<u8").view(np.uint8).reshape(*w.shape[:-1], -1)
    return np.unpackbits(bytes_, axis=-1, bitorder="little")[..., :n]


def sogrand_trace_patterns(code: Code, llr, max_q: int):
    """Device query order of one word: (rank masks [q, n] u8, c)."""
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    nm = (code.n + 63) // 64
    out = np.zeros((max_q, nm), dtype=np.uint64)
    cnt = C.c_int64(0)
    c = C.c_int32(0)
    _check(load().sogrand_trace_patterns(code.handle, llr.ctypes.data_as(C.c_void_p), int(max_q),
                                         out.ctypes.data_as(C.c_void_p), C.byref(cnt), C.byref(c)),
           "sogrand_trace_patterns")
    q = cnt.value
    return unpack_words(out[:q].view(np.int64), code.n), int(c.value)
