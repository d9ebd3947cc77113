"""GPU parity of sogrand_decode (the SOGRAND SISO kernel) against the oracle,
through the C ABI, on seeded BPSK/AWGN words shaped like the paper's
component decodings (Sec. V, VI): several codes, Eb/N0 points, list sizes,
a-priori inputs, ragged batch sizes that span many grid-stride passes, ties,
zeros, huge LLRs, non-finite inputs and the threshold rule."""
import numpy as np
import pytest

from gpu_common import compare_siso, llr_close
from workloads import awgn_words, ebch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_10737_gb300 as sg
    codes = {}

    def get(name):
        if name not in codes:
            lc = ebch(name)
            codes[name] = (lc, sg.Code.from_linear_code(lc), oracle_lib.OracleCode(lc))
        return codes[name]

    yield torch, sg, get
    for _, c, _ in codes.values():
        c.close()


def _run(env, oracle_lib, name, lch, la=None, L=4, cap=10**4, thr=0.0, what=""):
    torch, sg, get = env
    lc, c, oc = get(name)
    t_ch = torch.from_numpy(np.ascontiguousarray(lch, np.float32)).cuda()
    t_a = None if la is None else torch.from_numpy(np.ascontiguousarray(la, np.float32)).cuda()
    out = sg.sogrand_decode(c, t_ch, t_a, L=L, query_cap=cap, thr=thr)
    torch.cuda.synchronize()
    ref = oracle_lib.siso_batch(oc, lch, la, L=L, cap=cap, thr=thr)
    return lc, out, ref


@pytest.mark.parametrize("name,ebn0,W", [("ebch_8_4", 2.0, 300), ("ebch_16_11", 2.5, 700), ("ebch_32_26", 2.0, 1500),
                                         ("ebch_32_26", 4.0, 5203), ("ebch_64_57", 3.0, 1200),
                                         ("ebch_64_57", 5.0, 2000), ("ebch_64_51", 3.0, 600),
                                         ("ebch_128_120", 4.0, 400)])
@pytest.mark.parametrize("L", [1, 4])
def test_siso_parity_channel_only(env, oracle_lib, name, ebn0, W, L):
    lc = ebch(name)
    _, _, lch = awgn_words(lc, W, ebn0, seed=1000 + W)
    lc, out, ref = _run(env, oracle_lib, name, lch, L=L, what=f"{name} {ebn0}dB L={L}")
    compare_siso(lc, out, ref, f"{name} {ebn0}dB L={L}")


@pytest.mark.parametrize("name", ["ebch_32_26", "ebch_64_57", "ebch_128_120"])
def test_siso_parity_with_apriori(env, oracle_lib, name):
    """Later turbo half iterations: lambda = L_Ch + L_A with L_A agreeing with the codeword
    most of the time and large in magnitude."""
    lc = ebch(name)
    W = 800
    _, X, lch = awgn_words(lc, W, 3.0, seed=77)
    rng = np.random.default_rng(5)
    sgn = 1.0 - 2.0 * X
    flip = rng.random(X.shape) < 0.03
    mag = rng.uniform(2.0, 25.0, X.shape)
    la = (np.where(flip, -sgn, sgn) * mag).astype(np.float32)
    lc, out, ref = _run(env, oracle_lib, name, lch, la, L=4, what=f"{name} a-priori")
    compare_siso(lc, out, ref, f"{name} a-priori")


def test_siso_huge_llrs_use_extended_range(env, oracle_lib):
    """|lambda| in the hundreds: every mass underflows FP32; the extended-range
    remainder must still match the FP64 oracle."""
    lc = ebch("ebch_64_57")
    W = 300
    _, X, lch = awgn_words(lc, W, 3.0, seed=78)
    rng = np.random.default_rng(6)
    la = ((1.0 - 2.0 * X) * rng.uniform(100.0, 400.0, X.shape)).astype(np.float32)
    la[:, :3] *= -0.001  # a few unreliable bits
    lc, out, ref = _run(env, oracle_lib, "ebch_64_57", lch, la, L=4, what="huge")
    compare_siso(lc, out, ref, "huge")


@pytest.mark.parametrize("name", ["ebch_16_11", "ebch_64_57"])
def test_siso_ties_and_zeros(env, oracle_lib, name):
    lc = ebch(name)
    W = 500
    _, _, lch = awgn_words(lc, W, 2.5, seed=79)
    lch = np.round(lch * 2.0) / 2.0  # many exact ties, some exact zeros
    lch[0] = 0.0
    lch[1] = 1.0
    lch[2, ::2] = -0.0
    lc, out, ref = _run(env, oracle_lib, name, lch.astype(np.float32), L=4, what="ties")
    compare_siso(lc, out, ref, "ties")


@pytest.mark.parametrize("name", ["ebch_32_26", "ebch_64_57", "ebch_128_120"])
def test_siso_near_ties_in_the_last_mantissa_bits(env, oracle_lib, name):
    """Reliabilities that differ only in their last few mantissa bits, mostly
    with the larger one at the lower bit index (the rank order of Sec. III-B,
    ties by index, must follow the exact values): the kernel sorts on keys
    that keep |lambda| without its low mantissa bits, so these words take its
    exact second sort.  The pairs sit among the least reliable bits, whose
    ranks the first queries use, so a wrong order changes queries and lists."""
    lc = ebch(name)
    W, n = 600, lc.n
    _, _, lch = awgn_words(lc, W, 3.0, seed=83)
    mag = np.abs(lch).astype(np.float32)
    bits = mag.view(np.uint32) & np.uint32(0xFFFFFF00)  # low 8 mantissa bits cleared
    rng = np.random.default_rng(9)
    for w in range(W):
        low = np.argsort(mag[w], kind="stable")[: n // 2]
        pairs = rng.permutation(low)[: 2 * (len(low) // 4)].reshape(-1, 2)
        for i, j in pairs:
            i, j = min(i, j), max(i, j)
            bits[w, j] = bits[w, i]
            d = np.uint32(rng.integers(1, 32))  # stays below every key's dropped bits
            u = rng.random()
            if u < 0.7:
                bits[w, i] += d  # larger value at the lower index: against the index order
            elif u < 0.9:
                bits[w, j] += d  # with the index order
            # else: an exact tie, broken by the index
    lch2 = np.where(lch < 0, -1.0, 1.0).astype(np.float32) * bits.view(np.float32)
    lc, out, ref = _run(env, oracle_lib, name, lch2, L=4, what=f"{name} near ties")
    compare_siso(lc, out, ref, f"{name} near ties")


def test_siso_small_caps_empty_lists_and_list16(env, oracle_lib):
    lc = ebch("ebch_32_26")
    _, _, lch = awgn_words(lc, 700, 1.5, seed=80)
    for cap, L in ((1, 4), (5, 4), (37, 2), (20000, 16)):
        lc, out, ref = _run(env, oracle_lib, "ebch_32_26", lch, L=L, cap=cap, what=f"cap={cap}")
        compare_siso(lc, out, ref, f"cap={cap} L={L}")
        if cap == 1:
            assert (ref["list_count"] == 0).any()


def test_siso_nonfinite_inputs_flagged(env, oracle_lib):
    torch, sg, get = env
    lc, c, oc = get("ebch_32_26")
    _, _, lch = awgn_words(lc, 40, 3.0, seed=81)
    lch[3, 5] = np.nan
    lch[7, 0] = np.inf
    lch[9, 31] = -np.inf
    out = sg.sogrand_decode(c, torch.from_numpy(lch).cuda(), L=4, query_cap=1000)
    q = out["queries"].cpu().numpy()
    assert (q[[3, 7, 9]] == -1).all() and (q[[0, 1, 2, 4, 5, 6, 8]] > 0).all()
    assert (out["list_count"].cpu().numpy()[[3, 7, 9]] == 0).all()
    assert (out["p_miss"].cpu().numpy()[[3, 7, 9]] == 1.0).all()
    ref = oracle_lib.siso_batch(oc, lch[:3], L=4, cap=1000)
    assert (q[:3] == ref["queries"]).all()


def test_siso_threshold_rule(env, oracle_lib):
    """thr > 0 stops at the first list size with P(not in list) < thr.  The
    decision compares an FP32 estimate (GPU) with an FP64 one (oracle), so
    words whose oracle P(miss) lies within 1% of thr may legitimately differ."""
    lc = ebch("ebch_64_57")
    W = 1500
    _, _, lch = awgn_words(lc, W, 4.0, seed=82)
    thr = 1e-3
    lc, out, ref = _run(env, oracle_lib, "ebch_64_57", lch, L=4, thr=thr, what="thr")
    q = out["queries"].cpu().numpy()
    same = q == ref["queries"]
    assert same.mean() > 0.99
    for i in np.nonzero(~same)[0]:
        # the deciding P(miss) must be near the threshold on one side or the other
        k = min(ref["list_count"][i], out["list_count"].cpu().numpy()[i])
        r = oracle_lib.siso(oracle_lib.OracleCode(lc), lch[i], L=max(k, 1), cap=10**4)
        assert abs(r["pmiss"] - thr) < 0.01 * thr, (i, r["pmiss"])
    idx = np.nonzero(same)[0]
    assert llr_close(out["llr_app"].cpu().numpy()[idx], ref["lapp"][idx]).all()


def test_trace_order_matches_oracle(env, oracle_lib):
    torch, sg, get = env
    rng = np.random.default_rng(9)
    for name in ("ebch_16_11", "ebch_32_26", "ebch_64_57", "ebch_64_51", "ebch_128_120"):
        lc, c, oc = get(name)
        n = lc.n
        for trial in range(6):
            lam = (rng.normal(0, 1, n) * [0.5, 3.0, 8.0][trial % 3]).astype(np.float32)
            if trial == 5:
                lam = np.round(lam)
            masks, cdev = sg.sogrand_trace_patterns(c, lam, 3000)
            absl = np.sort(np.abs(lam))
            assert cdev == oracle_lib.one_line_c(absl, n)
            par = int((lam < 0).sum() & 1)
            ranks, _, _ = oracle_lib.trace(n, cdev, par, 3000)
            np.testing.assert_array_equal(masks, ranks, err_msg=f"{name} trial {trial}")


@pytest.mark.parametrize("name,ebn0,W,L", [("ebch_16_11", 2.0, 700, 5), ("ebch_32_26", 2.0, 1500, 5),
                                           ("ebch_64_57", 2.0, 1200, 5), ("ebch_64_51", 3.0, 400, 2),
                                           ("ebch_128_120", 4.0, 300, 1)])
def test_forney_parity(env, oracle_lib, name, ebn0, W, L):
    """Forney's list-only normalisation (eq. missingterm) against the oracle's
    reading 2: same search, APPs over the list, infinite L_APP on unanimous bits."""
    torch, sg, get = env
    lc, c, _ = get(name)
    _, _, lch = awgn_words(lc, W, ebn0, seed=2000 + W)
    out = sg.sogrand_decode(c, torch.from_numpy(lch).cuda(), L=L, query_cap=10**4, forney=True)
    torch.cuda.synchronize()
    ref = oracle_lib.siso_batch(oracle_lib.OracleCode(lc, reading=2), lch, L=L, cap=10**4)
    compare_siso(lc, out, ref, f"Forney {name} {ebn0}dB L={L}")
    pm = out["p_miss"].cpu().numpy()
    cnt = out["list_count"].cpu().numpy()
    assert (pm[cnt > 0] == 0).all() and (pm[cnt == 0] == 1).all()
    assert sg._lib.load().sogrand_decode_forney(c.handle, 1, None, None, 4, 10, *([None] * 8), None) == 1  # EINVAL
