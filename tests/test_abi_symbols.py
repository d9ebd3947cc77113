"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/sogrand.h declares; argument errors are reported before any
CUDA call, so they are checked here without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sogrand.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_10737_gb300 import build
    build.build()
    from paper_2310_10737_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"sogrand_code_create", "sogrand_decode", "product_decode", "sogrand_trace_patterns"} <= set(names)
    for nm in names:
        assert hasattr(lib, nm), nm


def test_argument_errors_without_gpu(lib):
    from paper_2310_10737_gb300 import _lib
    h = C.c_void_p()
    H = np.ones((1, 8), np.uint8)
    # n out of range, k >= n, entries not 0/1, even flag on a non-even code
    assert lib.sogrand_code_create(200, 100, H.ctypes.data_as(C.c_void_p), 1, C.byref(h)) == _lib.EINVAL
    assert lib.sogrand_code_create(8, 8, H.ctypes.data_as(C.c_void_p), 1, C.byref(h)) == _lib.EINVAL
    bad = np.full((1, 8), 2, np.uint8)
    assert lib.sogrand_code_create(8, 7, bad.ctypes.data_as(C.c_void_p), 0, C.byref(h)) == _lib.EINVAL
    odd = np.zeros((1, 8), np.uint8)
    odd[0, 0] = 1
    assert lib.sogrand_code_create(8, 7, odd.ctypes.data_as(C.c_void_p), 1, C.byref(h)) == _lib.EINVAL
    assert lib.sogrand_code_create(8, 7, None, 1, C.byref(h)) == _lib.EINVAL
    assert lib.sogrand_decode(None, 1, None, None, 4, 10, 0.0, *([None] * 8), None) == _lib.EINVAL
    assert lib.product_decode(None, None, 1, None, 4, 10, 0.0, 0.5, 4, None, None, None, None, None) == _lib.EINVAL
    assert lib.product_decode_mixed(0, None, 4, 10, 0.0, 0.5, 4, None, None) == _lib.EINVAL
    assert lib.product_decode_mixed(17, (_lib.FrameGroup * 17)(), 4, 10, 0.0, 0.5, 4, None, None) == _lib.EINVAL
    assert lib.sogrand_int_peak(0, None, None, None) == _lib.EINVAL
    assert lib.sogrand_strerror(_lib.EUNSUPPORTED).decode() == "unsupported configuration"
