"""Bounded device-side waits of the batched decoder (failure detection without
a GPU fault).

The persistent kernel has two waits: a warp waits for work on the device-side
frame-half list, and a warp waits for its block's remaining-mass lock.  Both
are bounded (sogrand_set_wait_limits).  Each test makes one wait run out on
purpose, with nothing faulting and nothing hanging:

* queue wait: a limit of 0 makes the first warp that finds no work give up
  (in a batch whose frames need more than one half, warps past the first
  half's tickets always wait for frames to be re-queued);
* lock wait: every block starts with its lock taken, as if a warp held it and
  never let go (a flag that nothing clears), and a limit of 16 polls.

The call must return SOGRAND_ETIMEOUT within seconds, and the context must stay
usable: with the default limits restored the same batch decodes exactly as
the plain form decodes it.
"""
import time

import numpy as np
import pytest

from workloads import awgn_frames, ebch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_10737_gb300 as sg
    yield torch, sg
    sg.sogrand_set_wait_limits(sg.DEFAULT_QUEUE_WAIT_US, sg.DEFAULT_LOCK_POLLS, 0)


def _decode(sg, c, d, persistent):
    return sg.product_decode(c, d, L=4, query_cap=10**4, alpha=0.5, max_iter=20, persistent=persistent)


def _expect_timeout_then_recover(env, code_name, F, ebn0, limits):
    torch, sg = env
    code = ebch(code_name)
    _, _, lch = awgn_frames(code, F, ebn0, seed=77)
    c = sg.Code.from_linear_code(code)
    d = torch.from_numpy(lch).cuda()
    ref = _decode(sg, c, d, persistent=False)
    torch.cuda.synchronize()
    assert (ref["half_iters"].cpu().numpy() > 1).any()  # some frame needs a second half
    sg.sogrand_set_wait_limits(*limits)
    try:
        t = time.perf_counter()
        with pytest.raises(sg.SograndError) as ei:
            _decode(sg, c, d, persistent=True)
        dt = time.perf_counter() - t
    finally:
        sg.sogrand_set_wait_limits(sg.DEFAULT_QUEUE_WAIT_US, sg.DEFAULT_LOCK_POLLS, 0)
    assert ei.value.code == 4, ei.value  # SOGRAND_ETIMEOUT
    assert dt < 30.0
    # the context is still usable and the batched form is correct again
    got = _decode(sg, c, d, persistent=True)
    torch.cuda.synchronize()
    for k in ("bits", "half_iters", "status", "queries"):
        np.testing.assert_array_equal(got[k].cpu().numpy(), ref[k].cpu().numpy(), err_msg=k)
    c.close()


def test_queue_wait_runs_out(env):
    _expect_timeout_then_recover(env, "ebch_32_26", 3000, 2.5, (0, -1, -1))


def test_remaining_mass_lock_wait_runs_out(env):
    # eBCH(64,51) words often need the exact remaining-mass sum (the block's lock)
    _expect_timeout_then_recover(env, "ebch_64_51", 400, 3.0, (-1, 16, 1))


def test_wait_limit_arguments(env):
    torch, sg = env
    with pytest.raises(sg.SograndError):
        sg.sogrand_set_wait_limits(1 << 40, -1, -1)
    with pytest.raises(sg.SograndError):
        sg.sogrand_set_wait_limits(-1, -1, 2)
    sg.sogrand_set_wait_limits(-1, -1, -1)  # keeps everything
