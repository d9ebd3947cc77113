"""Pins of the oracle's block turbo decoder of product codes (Sec. VI, Fig. turboDec).

* a noiseless frame is accepted after the first (row) half iteration;
* errors confined to distinct rows, each a single weak flip, are fixed by the
  row half alone, so decoding stops after one half iteration;
* a reported success is a product codeword (independent syndrome check on
  every row and column);
* the iteration cap is honoured and reported;
* BLER falls with Eb/N0 and the "parallelized" query count (sum over halves of
  the per-half maximum, Sec. VI) never exceeds the serial count.
"""
import numpy as np

from workloads import awgn_frames, ebch


def test_noiseless_frame_stops_after_first_half(oracle_lib):
    code = ebch("ebch_16_11")
    oc = oracle_lib.OracleCode(code)
    rng = np.random.default_rng(0)
    U = rng.integers(0, 2, (1, 11, 11), dtype=np.uint8)
    X = code.product_encode(U)[0]
    lch = (8.0 * (1.0 - 2.0 * X)).astype(np.float32)
    r = oracle_lib.product(oc, lch, L=4, cap=1000, max_iter=4)
    assert r["status"] == 0 and r["half_iters"] == 1
    assert (r["bits"] == X).all()


def test_single_errors_in_rows_fixed_by_first_half(oracle_lib):
    code = ebch("ebch_32_26")
    oc = oracle_lib.OracleCode(code)
    rng = np.random.default_rng(1)
    U = rng.integers(0, 2, (1, 26, 26), dtype=np.uint8)
    X = code.product_encode(U)[0]
    lch = (1.0 - 2.0 * X).astype(np.float32) * rng.uniform(4.0, 9.0, X.shape).astype(np.float32)
    for row in range(0, 32, 3):
        j = int(rng.integers(0, 32))
        lch[row, j] = -0.3 * np.sign(lch[row, j])
    r = oracle_lib.product(oc, lch, L=4, cap=10**4, max_iter=4)
    assert r["status"] == 0 and r["half_iters"] == 1 and (r["bits"] == X).all()


def test_success_means_product_codeword_and_caps(oracle_lib):
    code = ebch("ebch_16_11")
    oc = oracle_lib.OracleCode(code)
    U, X, L = awgn_frames(code, 60, 2.0, seed=5)
    res = oracle_lib.product_batch(oc, L, L=4, cap=1000, alpha=0.5, max_iter=3)
    assert (res["half_iters"] >= 1).all() and (res["half_iters"] <= 6).all()
    for f in range(60):
        B = res["bits"][f]
        valid = not code.syndrome(B).any() and not code.syndrome(B.T).any()
        assert valid == (res["status"][f] == 0)
        if res["status"][f] == 1:
            assert res["half_iters"][f] == 6
    assert (res["par_queries"] <= res["queries"]).all()
    assert (res["par_queries"] * code.n >= res["queries"]).all()


def test_bler_falls_with_snr(oracle_lib):
    code = ebch("ebch_16_11")
    oc = oracle_lib.OracleCode(code)
    bler = []
    for ebn0 in (1.0, 3.0):
        U, X, L = awgn_frames(code, 300, ebn0, seed=6)
        res = oracle_lib.product_batch(oc, L, L=4, cap=2000, alpha=0.5, max_iter=10)
        err = (res["bits"] != X).reshape(300, -1).any(axis=1)
        bler.append(err.mean())
    assert bler[0] > 0.1 and bler[1] < 0.02


def test_non_square_product_code(oracle_lib):
    """Product of different row and column codes (an n_col x n_row frame):
    rows are decoded with the row code, columns with the column code, and a
    frame succeeds iff every row and every column is a codeword of its code."""
    from workloads import awgn_frames, ebch
    r, c = ebch("ebch_32_26"), ebch("ebch_16_11")
    orc, occ = oracle_lib.OracleCode(r), oracle_lib.OracleCode(c)
    U, X, L = awgn_frames(r, 24, 3.0, seed=41, col_code=c)
    assert X.shape == (24, 16, 32)
    res = oracle_lib.product_batch(orc, L, col=occ, L=4, cap=10**4, alpha=0.5, max_iter=10)
    for f in range(24):
        B = res["bits"][f]
        ok = not r.syndrome(B).any() and not c.syndrome(B.T).any()
        assert ok == (res["status"][f] == 0)
    assert (res["status"] == 0).mean() > 0.8
    # noiseless: one half suffices
    clean = (8.0 * (1.0 - 2.0 * X[:2])).astype(np.float32)
    res0 = oracle_lib.product_batch(orc, clean, col=occ, max_iter=4)
    assert (res0["half_iters"] == 1).all() and (res0["bits"] == X[:2]).all()
    # a square code through the two-code path equals the one-code path
    Us, Xs, Ls = awgn_frames(c, 6, 2.5, seed=42)
    a = oracle_lib.product_batch(occ, Ls, max_iter=6)
    b = oracle_lib.product_batch(occ, Ls, max_iter=6, col=occ)
    for k in ("bits", "half_iters", "status", "queries", "par_queries"):
        np.testing.assert_array_equal(a[k], b[k])
