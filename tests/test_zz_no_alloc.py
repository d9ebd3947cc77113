"""product_decode_noalloc: product decoding for callers that cannot allocate
device memory (a fixed memory budget, or no allocation allowed on a stream
other work depends on).  Its scratch is one fixed device array inside the
library; the paper has no counterpart.

The entry point is called through the C ABI and must give exactly what
product_decode gives (the same kernels: bit-exact frames, half iterations,
status and query counts), on two calls in a row with different batches, so a
stale array from the first call would show in the second.  It must also
refuse batches larger than the array (also frame counts whose scratch size
would overflow), query caps its tables do not cover and row and column codes
that differ, writing nothing.  This file is collected last so that a failure here leaves
every other test already run; it passes alone and after the others.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import awgn_frames, ebch

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20  # SOGRAND_NOALLOC_SCRATCH_BYTES in include/sogrand.h


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_10737_gb300 as sg
    lib = sg.load()
    vp = C.c_void_p
    lib.product_decode_noalloc.argtypes = [vp, vp, C.c_int64, vp, C.c_int, C.c_int64, C.c_float, C.c_float, C.c_int,
                                           vp, vp, vp, vp, vp]
    lib.product_decode_noalloc.restype = C.c_int
    return torch, sg, lib


def _noalloc(env, code_h, lch, L=4, cap=10**4, alpha=0.5, max_iter=4, col_h=None, n_frames=None):
    torch, sg, lib = env
    F, n, _ = lch.shape
    dev = lch.device
    out = dict(bits=torch.full((F, (n * n + 7) // 8), 0xA5, dtype=torch.uint8, device=dev),
               half_iters=torch.full((F,), -7, dtype=torch.int32, device=dev),
               status=torch.full((F,), 9, dtype=torch.uint8, device=dev),
               queries=torch.full((F,), -5, dtype=torch.int64, device=dev))
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.product_decode_noalloc(code_h, code_h if col_h is None else col_h, F if n_frames is None else n_frames,
                                    C.c_void_p(lch.data_ptr()), L, cap, 0.0, alpha, max_iter,
                                    C.c_void_p(out["bits"].data_ptr()), C.c_void_p(out["half_iters"].data_ptr()),
                                    C.c_void_p(out["status"].data_ptr()), C.c_void_p(out["queries"].data_ptr()), s)
    torch.cuda.synchronize()
    return rc, {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_matches_product_decode_on_two_calls(env):
    torch, sg, lib = env
    code = ebch("ebch_32_26")
    c = sg.Code.from_linear_code(code)
    batches = [awgn_frames(code, 150, 2.75, seed=900)[2], awgn_frames(code, 97, 3.5, seed=901)[2]]
    for i, lch in enumerate(batches):
        d = torch.from_numpy(lch).cuda()
        ref = sg.product_decode(c, d, L=4, query_cap=10**4, alpha=0.5, max_iter=4)
        torch.cuda.synchronize()
        rc, got = _noalloc(env, c.handle, d)
        assert rc == 0, sg.strerror(rc)
        for key in ("bits", "half_iters", "status", "queries"):
            np.testing.assert_array_equal(got[key], ref[key].cpu().numpy(), err_msg=f"call {i}: {key}")
        assert (got["half_iters"] >= 1).all()
    c.close()


def test_noalloc_refuses_oversized_batches_and_uncovered_caps(env):
    torch, sg, lib = env
    code = ebch("ebch_64_57")
    c = sg.Code.from_linear_code(code)
    n = code.n
    per_frame = 4 * n * n + 8 * n * 1 + 16
    too_many = SCRATCH_BYTES // per_frame + 1
    lch = torch.zeros((too_many, n, n), dtype=torch.float32, device="cuda")
    rc, got = _noalloc(env, c.handle, lch)
    assert rc == 1  # SOGRAND_EINVAL
    assert (got["bits"] == 0xA5).all() and (got["half_iters"] == -7).all() and (got["queries"] == -5).all()
    small = torch.zeros((4, n, n), dtype=torch.float32, device="cuda")
    rc, got = _noalloc(env, c.handle, small, cap=10**4 + 1)  # the tables cover 10^4 only
    assert rc == 1 and (got["status"] == 9).all()
    # a frame count so large that the scratch size would wrap around 2^64
    rc, got = _noalloc(env, c.handle, small, n_frames=1 << 62)
    assert rc == 1 and (got["half_iters"] == -7).all() and (got["bits"] == 0xA5).all()
    # only the square product of one code: another column code is refused
    other = sg.Code.from_linear_code(ebch("ebch_64_51"))
    rc, got = _noalloc(env, c.handle, small, col_h=other.handle)
    assert rc == 5 and (got["queries"] == -5).all()  # SOGRAND_EUNSUPPORTED
    other.close()
    fits = SCRATCH_BYTES // per_frame - 4
    rc, got = _noalloc(env, c.handle, torch.full((fits, n, n), 5.0, dtype=torch.float32, device="cuda"), max_iter=1)
    assert rc == 0 and (got["status"] == 0).all() and (got["half_iters"] == 1).all()
    c.close()
