"""Pins of the oracle's SOGRAND SISO decoder (Sec. IV Corollary, Sec. V-B eq. LLRi).

Pins that do not re-use the oracle's own arithmetic:
* exhaustive enumeration on tiny codes (8,4) and (16,11): with the query cap
  at the size of the parity class (L above 2^k) every codeword is listed, the
  list-miss probability is 0, the list's APPs are the exact posterior
  (eq. formula:forney, Sec. II-C) and L_APP equals the exact bitwise APP by
  brute force over the codebook; the most probable list word is the ML word;
* the remaining (unqueried) mass equals a brute-force sum over all 2^n
  patterns minus the queried prefix (n = 16), for both readings;
* the list and the query count equal an independent scan of the query order
  with an independent membership test;
* APPs + P(not in list) = 1; L_E = L_APP - lambda; the threshold rule stops
  at the first list size whose P(not in list) is below thr;
* statistical calibration of P(not in list) (the paper's Fig. list_BLER):
  the empirical list-miss rate matches the prediction in every bin for the
  parity-class reading, and the literal reading overestimates it.
"""
import math

import numpy as np
import pytest

from workloads import awgn_words, ebch


def _oc(oracle_lib, name, **kw):
    return oracle_lib.OracleCode(ebch(name), **kw)


def _codebook(code):
    k = code.k
    U = ((np.arange(2 ** k)[:, None] >> np.arange(k)) & 1).astype(np.uint8)
    return code.encode(U)


def _exact_bitwise_llr(lam, book):
    # f(r|c) proportional to prod_j exp((1 - 2 c_j) lambda_j / 2)
    s = ((1.0 - 2.0 * book.astype(np.float64)) * lam[None, :]).sum(axis=1) / 2.0
    m = s.max()
    w = np.exp(s - m)
    out = np.empty(lam.size)
    for i in range(lam.size):
        a0 = w[book[:, i] == 0].sum()
        a1 = w[book[:, i] == 1].sum()
        out[i] = math.log(a0) - math.log(a1)
    return out, book[np.argmax(s)]


@pytest.mark.parametrize("name,ebn0", [("ebch_8_4", 0.0), ("ebch_8_4", 3.0), ("ebch_16_11", 1.0),
                                       ("ebch_16_11", 4.0)])
def test_exhaustive_list_gives_exact_app(oracle_lib, name, ebn0):
    code = ebch(name)
    oc = oracle_lib.OracleCode(code)
    book = _codebook(code)
    _, X, L = awgn_words(code, 12, ebn0, seed=21)
    rng = np.random.default_rng(1)
    for i in range(L.shape[0]):
        la = (rng.normal(0, 1.5, code.n) if i % 3 == 0 else np.zeros(code.n)).astype(np.float32)
        # L = 2^k + 1 is never reached, so the whole parity class is queried
        r = oracle_lib.siso(oc, L[i], la, L=2 ** code.k + 1, cap=2 ** (code.n - 1))
        lam = (L[i] + la).astype(np.float32).astype(np.float64)
        assert r["list_count"] == 2 ** code.k
        assert r["pmiss"] == 0.0 and r["log_r"] == -np.inf
        words = {tuple(w) for w in r["list_words"]}
        assert words == {tuple(w) for w in book}
        exact, ml = _exact_bitwise_llr(lam, book)
        np.testing.assert_allclose(r["lapp"], exact, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(r["lext"], exact - lam, rtol=1e-10, atol=1e-10)
        assert tuple(r["list_words"][np.argmax(r["list_app"])]) == tuple(ml)
        assert abs(r["list_app"].sum() - 1.0) < 1e-12


def test_exhaustive_literal_reading_is_not_exact(oracle_lib):
    """The literal reading keeps the other parity class in the remaining mass,
    so even an exhaustive search reports a nonzero miss probability."""
    code = ebch("ebch_8_4")
    oc = oracle_lib.OracleCode(code, reading=1)
    _, X, L = awgn_words(code, 4, 2.0, seed=2)
    for i in range(4):
        r = oracle_lib.siso(oc, L[i], L=17, cap=128)
        assert r["list_count"] == 16 and r["pmiss"] > 0


def _bruteforce_remaining(lam, c, cls, q, n, oracle_lib):
    """sum over patterns of the class not among the first q queries of prod exp(-|lam|)."""
    order = np.lexsort((np.arange(n), np.abs(lam).astype(np.float32)))
    absl = np.abs(lam).astype(np.float32).astype(np.float64)[order]
    ranks, cost, w = oracle_lib.trace(n, c, cls, 2 ** n)
    keys = ranks.astype(np.int64) @ (1 << np.arange(n, dtype=np.int64))
    queried = set(keys[:q].tolist())
    allk = np.arange(2 ** n, dtype=np.int64)
    bits = ((allk[:, None] >> np.arange(n)) & 1).astype(np.float64)
    pop = bits.sum(axis=1).astype(int)
    sel = np.ones(2 ** n, bool) if cls < 0 else (pop & 1) == cls
    sel &= ~np.isin(allk, np.fromiter(queried, np.int64))
    vals = np.exp(-(bits[sel] @ absl))
    return math.fsum(vals.tolist())


@pytest.mark.parametrize("reading", [0, 1])
def test_remaining_mass_equals_bruteforce_complement(oracle_lib, reading):
    code = ebch("ebch_16_11")
    oc = oracle_lib.OracleCode(code, reading=reading)
    _, X, L = awgn_words(code, 24, [1.0, 3.0, 6.0, 9.0] * 6, seed=8)
    rng = np.random.default_rng(3)
    n = code.n
    for i in range(L.shape[0]):
        la = (rng.normal(0, 4.0, n) if i % 2 else np.zeros(n)).astype(np.float32)
        for Lsz, cap in ((1, 1000), (4, 1000), (2, 7), (4, 60)):
            r = oracle_lib.siso(oc, L[i], la, L=Lsz, cap=cap)
            lam = (L[i] + la).astype(np.float32).astype(np.float64)
            cls = r["parity"]
            rem = _bruteforce_remaining(lam, r["c"], cls, r["queries"], n, oracle_lib)
            if reading == 1:
                # literal reading: every pattern of the other class is unqueried too
                order = np.abs(lam)
                tp = np.prod(1 + np.exp(-order))
                tm = np.prod(1 - np.exp(-order))
                rem += 0.5 * (tp - tm) if cls == 0 else 0.5 * (tp + tm)
            assert math.isclose(r["log_r"], math.log(rem), rel_tol=0, abs_tol=1e-10), (i, Lsz, cap)


def _scan_list(code, lam, c, cls, L, cap, oracle_lib):
    n = code.n
    order = np.lexsort((np.arange(n), np.abs(lam)))
    y = (lam < 0).astype(np.uint8)
    ranks, _, _ = oracle_lib.trace(n, c, cls, cap)
    z = np.zeros((ranks.shape[0], n), np.uint8)
    z[:, order] = ranks  # rank r-1 -> bit order[r-1]
    x = z ^ y[None, :]
    ok = ~code.syndrome(x).any(axis=1)
    hits = np.nonzero(ok)[0][:L]
    q = int(hits[-1]) + 1 if len(hits) == L else ranks.shape[0]
    return x[hits], hits + 1, q


@pytest.mark.parametrize("name,ebn0", [("ebch_32_26", 3.0), ("ebch_64_57", 3.0), ("ebch_64_51", 4.0),
                                       ("ebch_128_120", 4.0)])
def test_list_and_query_count_match_independent_scan(oracle_lib, name, ebn0):
    code = ebch(name)
    oc = oracle_lib.OracleCode(code)
    _, X, L = awgn_words(code, 10, ebn0, seed=4)
    for i in range(L.shape[0]):
        for Lsz in (1, 4):
            r = oracle_lib.siso(oc, L[i], L=Lsz, cap=3000)
            lam = L[i].astype(np.float32)
            words, qs, q = _scan_list(code, lam, r["c"], r["parity"], Lsz, 3000, oracle_lib)
            assert r["queries"] == q
            assert r["list_count"] == len(qs)
            np.testing.assert_array_equal(r["list_words"], words)
            np.testing.assert_array_equal(r["list_q"], qs)
            flips = r["list_words"] ^ (lam < 0)[None, :]
            np.testing.assert_allclose(r["list_logp"], -(flips * np.abs(lam.astype(np.float64))).sum(1),
                                       rtol=1e-12, atol=1e-9)
            if r["list_count"]:
                assert abs(r["list_app"].sum() + r["pmiss"] - 1.0) < 1e-12
            np.testing.assert_allclose(r["lext"], r["lapp"] - lam.astype(np.float64), atol=1e-12)
            assert (r["hard"] == (r["lapp"] < 0)).all()


def test_remaining_mass_matches_paper_literal_difference_when_well_conditioned(oracle_lib):
    code = ebch("ebch_64_57")
    oc = oracle_lib.OracleCode(code)
    _, X, L = awgn_words(code, 60, 2.5, seed=9)
    checked = 0
    for i in range(L.shape[0]):
        r = oracle_lib.siso(oc, L[i], L=4, cap=10**4)
        if r["log_r"] - math.log(r["S"] + 1.0) > math.log(1e-6):
            assert abs(r["log_r"] - r["log_r_direct"]) < 1e-6
            checked += 1
    assert checked > 30


def test_single_word_corollary_and_empty_list(oracle_lib):
    code = ebch("ebch_32_26")
    oc = oracle_lib.OracleCode(code)
    _, X, L = awgn_words(code, 20, 2.0, seed=12)
    for i in range(20):
        r = oracle_lib.siso(oc, L[i], L=1, cap=10**4)
        if r["list_count"] == 1:
            p = math.exp(r["list_logp"][0])
            rphi = math.exp(r["log_r"] + r["log_phi"])
            assert math.isclose(r["list_app"][0], p / (p + rphi), rel_tol=1e-12)
        r0 = oracle_lib.siso(oc, L[i], L=4, cap=1)  # only the hard decision is tried
        if r0["list_count"] == 0:
            lam = L[i].astype(np.float64)
            assert r0["pmiss"] == 1.0 and (r0["lapp"] == lam).all() and (r0["lext"] == 0).all()
    lam = L[0].copy()
    lam[3] = np.nan
    assert oracle_lib.siso(oc, lam)["queries"] == -1


def test_threshold_rule_stops_at_first_small_list_miss(oracle_lib):
    code = ebch("ebch_32_26")
    oc = oracle_lib.OracleCode(code)
    _, X, L = awgn_words(code, 40, 3.5, seed=13)
    stopped = 0
    for i in range(40):
        r = oracle_lib.siso(oc, L[i], L=4, cap=10**4, thr=1e-3)
        h = r["list_count"]
        for j in range(1, h):
            assert oracle_lib.siso(oc, L[i], L=j, cap=10**4)["pmiss"] >= 1e-3
        if r["thr_stop"]:
            stopped += 1
            assert oracle_lib.siso(oc, L[i], L=h, cap=10**4)["pmiss"] < 1e-3
            assert r["pmiss"] < 1e-3
    assert stopped > 5


def _calibration(oracle_lib, reading, n_words=16000):
    code = ebch("ebch_32_26")
    oc = oracle_lib.OracleCode(code, reading=reading)
    _, X, L = awgn_words(code, n_words, 2.0, seed=77)
    res = oracle_lib.siso_batch(oc, L, L=4, cap=10**4)
    miss = np.array([not any((w == X[i]).all() for w in it["list_words"]) for i, it in enumerate(res["items"])])
    return res["pmiss"], miss


@pytest.mark.slow
def test_list_miss_probability_is_calibrated(oracle_lib):
    """Fig. list_BLER: predicted vs empirical list-BLER, L = 4, Eb/N0 = 2 dB."""
    pred, miss = _calibration(oracle_lib, 0)
    edges = 10.0 ** np.arange(-5, 0.01, 0.5)
    used = 0
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (pred >= lo) & (pred < hi)
        if sel.sum() < 200:
            continue
        expect = pred[sel].sum()
        got = miss[sel].sum()
        sd = math.sqrt(max(expect, 1.0))
        assert abs(got - expect) < 4.5 * sd + 0.1 * expect, (lo, got, expect)
        used += 1
    assert used >= 4
    # the overall miss rate agrees too, while the literal reading predicts far more misses
    assert abs(miss.sum() - pred.sum()) < 4.5 * math.sqrt(pred.sum()) + 0.05 * pred.sum()
    pred_a, miss_a = _calibration(oracle_lib, 1, 4000)
    assert pred_a.sum() > 1.5 * miss_a.sum()


@pytest.mark.parametrize("name,ebn0", [("ebch_8_4", 1.0), ("ebch_16_11", 2.0)])
def test_forney_reading_with_the_whole_codebook_is_exact(oracle_lib, name, ebn0):
    """Forney's approximation (eq. missingterm) drops the mass outside the
    list; when the list holds the whole codebook nothing is dropped and the
    APPs are the exact posterior (eq. formula:forney)."""
    code = ebch(name)
    oc = oracle_lib.OracleCode(code, reading=2)
    book = _codebook(code)
    _, X, L = awgn_words(code, 8, ebn0, seed=31)
    for i in range(L.shape[0]):
        r = oracle_lib.siso(oc, L[i], L=2 ** code.k + 1, cap=2 ** (code.n - 1))
        lam = L[i].astype(np.float64)
        assert r["list_count"] == 2 ** code.k and r["pmiss"] == 0.0
        exact, ml = _exact_bitwise_llr(lam, book)
        np.testing.assert_allclose(r["lapp"], exact, rtol=1e-10, atol=1e-10)
        assert tuple(r["list_words"][np.argmax(r["list_app"])]) == tuple(ml)


def test_forney_reading_normalises_over_the_list(oracle_lib):
    code = ebch("ebch_32_26")
    oc_f = oracle_lib.OracleCode(code, reading=2)
    oc_b = oracle_lib.OracleCode(code)
    _, X, L = awgn_words(code, 30, 2.0, seed=32)
    for i in range(30):
        f = oracle_lib.siso(oc_f, L[i], L=4, cap=10**4)
        b = oracle_lib.siso(oc_b, L[i], L=4, cap=10**4)
        # the same search: same list, same queries
        assert f["queries"] == b["queries"] and f["list_count"] == b["list_count"]
        if f["list_count"] == 0:
            continue
        assert f["pmiss"] == 0.0
        assert abs(f["list_app"].sum() - 1.0) < 1e-12
        # each Forney APP is SOGRAND's APP rescaled by 1 / (1 - P(miss))
        np.testing.assert_allclose(f["list_app"], b["list_app"] / (1.0 - b["pmiss"]), rtol=1e-9)
        # a bit on which every listed word agrees gets an infinite L_APP of that sign
        W = f["list_words"]
        unanimous = (W == W[0]).all(axis=0)
        assert np.isinf(f["lapp"][unanimous]).all()
        assert ((f["lapp"][unanimous] < 0) == (W[0][unanimous] == 1)).all()
        assert np.isfinite(f["lapp"][~unanimous]).all()
    f1 = oracle_lib.siso(oc_f, L[0], L=1, cap=10**4)
    if f1["list_count"] == 1:
        assert f1["list_app"][0] == 1.0
