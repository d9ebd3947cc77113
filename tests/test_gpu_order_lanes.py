"""The query order enumerated by the lanes (sogrand_code_order_source = 1)
against the oracle and against the order-table path.

1-line ORBGRAND (Sec. III-B) queries the patterns by increasing cost = rank
sum + c * weight; the patterns of one cost and weight are the partitions of
the rank sum into distinct parts <= n, in lexicographic order of the rank
vector.  The lanes unrank those partitions from subset counts instead of
reading the precomputed table, so the order, and with it every query count,
list and soft output, must be the same: bit-exact against the oracle in
queries and lists (the parity bar of the SISO), and identical in every output
to the table path in product decoding."""
import numpy as np
import pytest

from gpu_common import compare_siso
from workloads import awgn_frames, awgn_words, ebch

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


@pytest.mark.parametrize("name,ebn0,W,L,cap", [("ebch_8_4", 1.0, 300, 4, 10**4), ("ebch_16_11", 2.0, 700, 4, 10**4),
                                               ("ebch_32_26", 2.0, 1500, 4, 10**4),
                                               ("ebch_64_57", 3.0, 1200, 4, 10**4),
                                               ("ebch_64_51", 3.0, 500, 4, 10**4),
                                               ("ebch_128_120", 4.0, 400, 4, 10**4),
                                               ("ebch_64_57", 2.0, 300, 16, 10**5),
                                               ("ebch_32_26", 1.5, 700, 2, 37)])
def test_lanes_order_matches_oracle(env, oracle_lib, name, ebn0, W, L, cap):
    torch, sg = env
    lc = ebch(name)
    _, X, lch = awgn_words(lc, W, ebn0, seed=2000 + W)
    la = None
    if name == "ebch_64_57" and L == 4:  # a later half: large a-priori values, a few of them wrong
        rng = np.random.default_rng(11)
        sgn = 1.0 - 2.0 * X
        la = (np.where(rng.random(X.shape) < 0.03, -sgn, sgn) * rng.uniform(2.0, 25.0, X.shape)).astype(np.float32)
    c = sg.Code.from_linear_code(lc)
    c.reserve(cap)
    assert c.order_source() == 0
    assert c.order_source(1) == 1
    t_a = None if la is None else torch.from_numpy(la).cuda()
    out = sg.sogrand_decode(c, torch.from_numpy(lch).cuda(), t_a, L=L, query_cap=cap)
    torch.cuda.synchronize()
    c.close()
    ref = oracle_lib.siso_batch(oracle_lib.OracleCode(lc), lch, la, L=L, cap=cap)
    compare_siso(lc, out, ref, f"{name} lanes L={L} cap={cap}")


@pytest.mark.parametrize("name,ebn0,F,max_iter", [("ebch_32_26", 2.75, 300, 4), ("ebch_64_57", 2.75, 200, 20),
                                                  ("ebch_64_51", 3.0, 50, 8), ("ebch_128_120", 3.75, 24, 5)])
def test_lanes_order_equals_table_in_product_decoding(env, name, ebn0, F, max_iter):
    torch, sg = env
    code = ebch(name)
    _, _, lch = awgn_frames(code, F, ebn0, seed=700 + F)
    c = sg.Code.from_linear_code(code)
    d = torch.from_numpy(lch).cuda()
    outs = []
    for src in (0, 1, 0):
        c.order_source(src)
        o = sg.product_decode(c, d, L=4, query_cap=10**4, alpha=0.5, max_iter=max_iter, persistent=True)
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy() for k, v in o.items() if hasattr(v, "cpu")})
    c.close()
    for key in ("bits", "half_iters", "status", "queries", "par_queries", "weight_sum"):
        np.testing.assert_array_equal(outs[1][key], outs[0][key], err_msg=key)
        np.testing.assert_array_equal(outs[2][key], outs[0][key], err_msg=key)


def test_order_source_refuses_unknown_values(env):
    torch, sg = env
    c = sg.Code.from_linear_code(ebch("ebch_16_11"))
    with pytest.raises(sg.SograndError):
        c.order_source(2)
    assert c.order_source() == 0
    c.close()


def test_lanes_trace_matches_oracle_order(env, oracle_lib):
    """Pattern by pattern: the first 3000 queries the lanes enumerate (group
    found from the chunk's group starts, partition unranked from subset
    counts) equal the oracle's 1-line ORBGRAND order (Sec. III-B) and the
    order table's, for the parameter c and parity class of the word."""
    torch, sg = env
    rng = np.random.default_rng(19)
    for name in ("ebch_16_11", "ebch_32_26", "ebch_64_57", "ebch_64_51", "ebch_128_120"):
        lc = ebch(name)
        n = lc.n
        c = sg.Code.from_linear_code(lc)
        for trial in range(6):
            lam = (rng.normal(0, 1, n) * [0.5, 3.0, 8.0][trial % 3]).astype(np.float32)
            if trial == 5:
                lam = np.round(lam)
            c.order_source(0)
            table, c_tab = sg.sogrand_trace_patterns(c, lam, 3000)
            c.order_source(1)
            lanes, c_lanes = sg.sogrand_trace_patterns(c, lam, 3000)
            assert c_lanes == c_tab
            par = int((lam < 0).sum() & 1)
            ranks, _, _ = oracle_lib.trace(n, c_lanes, par, 3000)
            np.testing.assert_array_equal(lanes, ranks, err_msg=f"{name} trial {trial}")
            np.testing.assert_array_equal(lanes, table, err_msg=f"{name} trial {trial}")
        c.close()
