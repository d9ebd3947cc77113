"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare element by element.

Parity bar (the hot path's contract):
* bit-exact: query counts, list sizes, listed codewords and their order,
  pattern order (trace);
* hard decisions equal except near-ties |L_APP(oracle)| <= 1e-3 (counted);
* soft outputs |L_gpu - L_oracle| <= 1e-3 + 1e-4 |L_oracle| (same-sign
  infinities match); probabilities |p_gpu - p_oracle| <= 1e-4 + 1e-3 p_oracle.
"""
import numpy as np

LLR_ATOL, LLR_RTOL = 1e-3, 1e-4
P_ATOL, P_RTOL = 1e-4, 1e-3


def llr_close(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    inf = np.isinf(ref)
    ok = np.zeros(ref.shape, bool)
    ok[inf] = gpu[inf] == ref[inf]
    fin = ~inf
    ok[fin] = np.abs(gpu[fin] - ref[fin]) <= LLR_ATOL + LLR_RTOL * np.abs(ref[fin])
    return ok


def compare_siso(code, out, ref, what=""):
    """out: dict of CUDA tensors from sogrand_decode; ref: oracle.siso_batch result."""
    import paper_2310_10737_gb300 as sg
    n = code.n
    q = out["queries"].cpu().numpy()
    np.testing.assert_array_equal(q, ref["queries"], err_msg=f"{what}: query counts")
    cnt = out["list_count"].cpu().numpy()
    np.testing.assert_array_equal(cnt, ref["list_count"], err_msg=f"{what}: list sizes")
    words = sg.unpack_words(out["list_words"], n)
    for i, it in enumerate(ref["items"]):
        if it["list_count"]:
            np.testing.assert_array_equal(words[i, :it["list_count"]], it["list_words"],
                                          err_msg=f"{what}: list of word {i}")
    lapp = out["llr_app"].cpu().numpy()
    ok = llr_close(lapp, ref["lapp"])
    bad = np.argwhere(~ok)
    assert ok.all(), f"{what}: {len(bad)} L_APP outside tolerance, first {bad[:3].tolist()} " \
                     f"gpu {lapp[tuple(bad[0])] if len(bad) else None} ref {ref['lapp'][tuple(bad[0])] if len(bad) else None}"
    lext = out["llr_ext"].cpu().numpy()
    assert llr_close(lext, ref["lext"]).all(), f"{what}: L_E outside tolerance"
    hard = out["hard"].cpu().numpy()
    near = np.abs(ref["lapp"]) <= 1e-3
    assert (hard[~near] == ref["hard"][~near]).all(), f"{what}: hard decisions"
    pm = out["p_miss"].cpu().numpy().astype(np.float64)
    assert (np.abs(pm - ref["pmiss"]) <= P_ATOL + P_RTOL * ref["pmiss"]).all(), f"{what}: p_miss"
    app = out["list_app"].cpu().numpy().astype(np.float64)
    for i, it in enumerate(ref["items"]):
        k = it["list_count"]
        if k:
            assert (np.abs(app[i, :k] - it["list_app"]) <= P_ATOL + P_RTOL * it["list_app"]).all(), \
                f"{what}: list APP of word {i}"
    return int(near.sum())
