"""Pin of the oracle's extrinsic exchange between half iterations (Sec. VI,
steps 1/2 and Fig. turboDec; Sec. V-B for L_E).

With an exhaustive list (query cap = the whole parity class, L above 2^k)
SOGRAND's L_APP is the exact bitwise APP of the SISO input (eq.
formula:forney summed over the codebook), so the whole turbo chain can be
recomputed by brute force without any of the oracle's search or soft-output
code:

    lambda_1 = L_Ch                               (L_A = 0 in the first half)
    L_APP_h  = exact APP of each word of half h (rows when h is odd, columns
               when h is even) given lambda_h, by enumeration of the codebook
    L_E_h    = fl32(L_APP_h - lambda_h)           (lambda_h = L_Ch + L_A)
    lambda_{h+1} = fl32(L_Ch + fl32(alpha L_E_h))

Each half's L_APP recorded by the oracle must equal this chain.  A wrong
a-priori term (alpha L_APP instead of alpha L_E), an extrinsic that forgets to
subtract the a-priori part, a stale or missing exchange, or rows and columns
taken in the wrong order each move L_APP by O(1) from the second or third half
on, while rounding differences between the two computations stay near 1e-12
(and at one FP32 ulp of lambda when an L_E value sits on a rounding
boundary).
"""
import numpy as np
import pytest

from workloads import awgn_frames, ebch


def _codebook(code):
    k = code.k
    U = ((np.arange(2 ** k)[:, None] >> np.arange(k)) & 1).astype(np.uint8)
    return code.encode(U)


def _exact_app(lam_words, book):
    """Exact bitwise APP LLRs of every word (rows of lam_words) by enumeration:
    p(c | r) is proportional to prod_j exp((1 - 2 c_j) lambda_j / 2)."""
    lam = lam_words.astype(np.float64)
    sgn = 1.0 - 2.0 * book.astype(np.float64)          # [C, n]
    s = lam @ sgn.T / 2.0                               # [W, C]
    s -= s.max(axis=1, keepdims=True)
    w = np.exp(s)
    one = book.astype(np.float64)                       # [C, n]
    a1 = w @ one                                        # [W, n] mass of the codewords with bit i = 1
    a0 = w @ (1.0 - one)                                # and with bit i = 0 (both positive sums)
    return np.log(a0) - np.log(a1)


def _brute_force_chain(lch, book, alpha, halves):
    """Per half h = 1..halves: the exact L_APP of that half as a [n_col, n_row] array."""
    lch = lch.astype(np.float32)
    le = np.zeros_like(lch)
    out = []
    a32 = np.float32(alpha)
    for h in range(1, halves + 1):
        lam = (lch + (a32 * le).astype(np.float32)).astype(np.float32)
        rows = h % 2 == 1
        app = _exact_app(lam if rows else lam.T, book)
        if not rows:
            app = app.T
        out.append(app)
        le = (app - lam.astype(np.float64)).astype(np.float32)
    return out


@pytest.mark.parametrize("name,ebn0,frames,max_iter", [("ebch_8_4", 0.0, 24, 4), ("ebch_8_4", 1.5, 24, 4),
                                                        ("ebch_16_11", 1.0, 5, 3)])
def test_exchange_between_halves_matches_brute_force_chain(oracle_lib, name, ebn0, frames, max_iter):
    code = ebch(name)
    oc = oracle_lib.OracleCode(code)
    book = _codebook(code)
    _, X, lch = awgn_frames(code, frames, ebn0, seed=1700 + frames)
    L = 2 ** code.k + 1                  # never reached: every codeword of the class is listed
    cap = 2 ** (code.n - 1)              # the whole parity class
    deep = 0
    for f in range(frames):
        r = oracle_lib.product_trace(oc, lch[f], L=L, cap=cap, alpha=0.5, max_iter=max_iter)
        H = r["half_iters"]
        assert 1 <= H <= 2 * max_iter
        ref = _brute_force_chain(lch[f], book, 0.5, H)
        for h in range(H):
            got = r["lapp_trace"][h]
            assert np.isfinite(got).all()
            err = np.abs(got - ref[h])
            tol = 1e-6 + 1e-6 * np.abs(ref[h])
            assert (err <= tol).all(), (f"frame {f} half {h + 1}: max |dL_APP| {err.max():.3g}", name, ebn0)
        assert np.isnan(r["lapp_trace"][H:]).all()
        # the frame stopped exactly when the hard decision of the last half became a product codeword
        B = (ref[H - 1] < 0).astype(np.uint8)
        valid = not code.syndrome(B).any() and not code.syndrome(B.T).any()
        assert valid == (r["status"] == 0)
        np.testing.assert_array_equal(r["bits"], B)
        deep += H >= 3
    # the chain is exercised past the first exchange (half 3 uses an L_E that had an a-priori part)
    assert deep >= 2


def test_exchange_uses_alpha(oracle_lib):
    """alpha scales the a-priori input: two values of alpha give different second
    halves, each equal to its own brute-force chain."""
    code = ebch("ebch_8_4")
    oc = oracle_lib.OracleCode(code)
    book = _codebook(code)
    _, X, lch = awgn_frames(code, 6, 0.0, seed=1777)
    for f in range(6):
        seconds = []
        for alpha in (0.25, 0.9):
            r = oracle_lib.product_trace(oc, lch[f], L=17, cap=128, alpha=alpha, max_iter=2)
            if r["half_iters"] < 2:
                break
            ref = _brute_force_chain(lch[f], book, alpha, 2)
            np.testing.assert_allclose(r["lapp_trace"][1], ref[1], rtol=1e-6, atol=1e-6)
            seconds.append(r["lapp_trace"][1])
        if len(seconds) == 2:
            assert np.abs(seconds[0] - seconds[1]).max() > 1e-3
