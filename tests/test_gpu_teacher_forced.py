"""Teacher-forced parity of product decoding, every half iteration (Sec. VI).

The plain form records, for every half h, the extrinsic state L_E after it and
the query count of every word it decoded (product_decode_ex traces).  Half h
(h >= 2) decoded its words from lambda_h = fl32(L_Ch + fl32(alpha L_E_{h-1}))
with L_E_{h-1} the GPU's own FP32 state, so the oracle's SISO given exactly
that lambda_h must reproduce the half:

* bit-exact: the query count of every word (hence the stop point of the list
  search, the list size and the pattern order up to it);
* L_E within 1e-3 + 1e-4 |L_E| (FP32 kernel arithmetic against the FP64
  oracle; the same bar as the SISO tests);
* hard decisions, read as the sign of lambda_h + L_E, equal except near-ties
  |L_APP| <= 1e-3.

This checks the kernels' exchange (lambda assembly, orientation, L_E
bookkeeping) and their SISO at every half on realistic late-half inputs,
including the large LLRs of converging frames.  Workloads: the plain-method
configuration (eBCH(32,26)^2, 200 frames at 3.0 dB, 4 iterations) and
eBCH(64,57)^2 frames across the benchmark's Eb/N0 range.
"""
import numpy as np
import pytest

from gpu_common import LLR_ATOL, LLR_RTOL
from workloads import awgn_frames, ebch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_10737_gb300 as sg
    return torch, sg


def _check_halves(env, oracle_lib, code, lch, max_iter, what, alpha=0.5, L=4, cap=10**4):
    torch, sg = env
    n = code.n
    F = lch.shape[0]
    c = sg.Code.from_linear_code(code)
    o = sg.product_decode(c, torch.from_numpy(lch).cuda(), L=L, query_cap=cap, alpha=alpha, max_iter=max_iter,
                          trace=True)
    torch.cuda.synchronize()
    hi = o["half_iters"].cpu().numpy()
    le = o["le_trace"].cpu().numpy()
    wq = o["word_queries"].cpu().numpy()
    qf = o["queries"].cpu().numpy()
    bits = sg.unpack_bits(o["bits"], n)
    c.close()
    oc = oracle_lib.OracleCode(code)
    a32 = np.float32(alpha)
    checked_words = near = 0
    for h in range(1, int(hi.max()) + 1):
        fr = np.nonzero(hi >= h)[0]
        if h == 1:
            lam = lch[fr]
        else:
            lam = (lch[fr] + (a32 * le[h - 2, fr]).astype(np.float32)).astype(np.float32)
        rows = h % 2 == 1
        words = lam if rows else lam.transpose(0, 2, 1)            # [f, word, bit]
        gle = le[h - 1, fr] if rows else le[h - 1, fr].transpose(0, 2, 1)
        ref = oracle_lib.siso_batch(oc, np.ascontiguousarray(words.reshape(-1, n)), L=L, cap=cap)
        gq = wq[h - 1, fr, :n].reshape(-1)
        bad = np.nonzero(gq != ref["queries"])[0]
        assert bad.size == 0, (f"{what} half {h}: {bad.size} words with different query counts, first "
                               f"{bad[:4].tolist()} gpu {gq[bad[:4]].tolist()} oracle {ref['queries'][bad[:4]].tolist()}")
        g = gle.reshape(-1, n).astype(np.float64)
        r = ref["lext"]
        ok = np.abs(g - r) <= LLR_ATOL + LLR_RTOL * np.abs(r)
        assert ok.all(), (f"{what} half {h}: {int((~ok).sum())} L_E outside tolerance, worst "
                          f"{np.abs(g - r)[~ok].max():.3g}")
        lam_w = words.reshape(-1, n).astype(np.float64)
        tie = np.abs(ref["lapp"]) <= 1e-3
        hard_g = (lam_w + g) < 0
        assert (hard_g[~tie] == ref["hard"][~tie].astype(bool)).all(), f"{what} half {h}: hard decisions"
        checked_words += gq.size
        near += int(tie.sum())
    # the traces add up to the per-frame totals, and the final bits are the last half's decision
    tot = np.zeros(F, np.int64)
    for h in range(1, int(hi.max()) + 1):
        run = hi >= h
        tot[run] += wq[h - 1, run, :n].astype(np.int64).sum(axis=1)
    np.testing.assert_array_equal(tot, qf)
    for f in range(F):
        h = hi[f]
        lam = lch[f] if h == 1 else (lch[f] + (a32 * le[h - 2, f]).astype(np.float32)).astype(np.float32)
        dec = (lam.astype(np.float64) + le[h - 1, f]) < 0
        assert (dec == bits[f].astype(bool)).mean() > 0.999
    return checked_words, near, hi


def test_plain_method_configuration_every_half(env, oracle_lib):
    code = ebch("ebch_32_26")
    _, _, lch = awgn_frames(code, 200, 3.0, seed=1)
    words, near, hi = _check_halves(env, oracle_lib, code, lch, 4, "eBCH(32,26)^2 3.0 dB")
    assert (hi >= 2).sum() >= 100 and hi.max() >= 4
    assert near <= 1e-4 * words * code.n + 2


def test_benchmark_code_every_half(env, oracle_lib):
    code = ebch("ebch_64_57")
    F = 105
    snr = (2.5 + 0.25 * np.arange(7))[np.arange(F) % 7]
    _, _, lch = awgn_frames(code, F, snr, seed=2310)
    words, near, hi = _check_halves(env, oracle_lib, code, lch, 20, "eBCH(64,57)^2 2.5..4.0 dB")
    assert (hi >= 3).sum() >= 30 and hi.max() >= 10
    assert near <= 1e-4 * words * code.n + 2
