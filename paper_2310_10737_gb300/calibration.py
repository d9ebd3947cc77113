"""Soft-output calibration harness (arXiv 2310.10737, Sec. IV "Blockwise SO
accuracy", Fig. list_BLER; Sec. V "Bitwise SO accuracy").

Decodes seeded words on the GPU and bins the predicted probability of an
error against the observed rate:

* blockwise: the predicted list-BLER of the first L' listed words against
  the rate at which the transmitted codeword is not among them.  SOGRAND
  (list L = L') predicts it with P(not in list) of the Corollary; Forney's
  approximation (list L' + 1, APPs normalised over the list) predicts it with
  the APP of the (L' + 1)-th word (0 when the search stopped before finding
  it);
* bitwise: the predicted bit-error probability 1 / (1 + e^|L_APP|) against the
  rate at which the hard decision of L_APP differs from the transmitted bit.

A calibrated soft output follows predicted = empirical in every bin.
"""
from __future__ import annotations

import numpy as np

from ._lib import Code, sogrand_decode, unpack_words


def _bins(pred, err, edges, min_count):
    rows = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (pred >= lo) & (pred < hi)
        cnt = int(sel.sum())
        if cnt < min_count:
            continue
        rows.append({"lo": float(lo), "hi": float(hi), "count": cnt, "predicted": float(pred[sel].mean()),
                     "empirical": float(err[sel].mean()), "expected_errors": float(pred[sel].sum()),
                     "errors": int(err[sel].sum())})
    return rows


def list_bler_calibration(code: Code, llr, X, L: int = 4, query_cap: int = 10**4, edges=None,
                          min_count: int = 200) -> dict:
    """llr: [W, n] float32 CUDA tensor of channel LLRs; X: [W, n] transmitted
    codewords (numpy u8).  Returns the binned calibration of both methods."""
    if edges is None:  # half-decade bins; the first also takes predictions of exactly 0
        edges = 10.0 ** np.arange(-6.0, 0.01, 0.5)
        edges[0] = 0.0
        edges[-1] = 1.0 + 1e-9
    X = np.asarray(X, dtype=np.uint8)
    n = code.n

    def first_hits(out, depth):
        words = unpack_words(out["list_words"], n)[:, :depth, :]
        cnt = out["list_count"].cpu().numpy()
        found = (words == X[:, None, :]).all(axis=2) & (np.arange(depth)[None, :] < cnt[:, None])
        return found.any(axis=1)

    s = sogrand_decode(code, llr, L=L, query_cap=query_cap)
    pred_s = s["p_miss"].cpu().numpy().astype(np.float64)
    miss_s = ~first_hits(s, L)
    f = sogrand_decode(code, llr, L=L + 1, query_cap=query_cap, forney=True)
    app = f["list_app"].cpu().numpy().astype(np.float64)
    cnt = f["list_count"].cpu().numpy()
    pred_f = np.where(cnt > L, app[:, L], 0.0)
    miss_f = ~first_hits(f, L)
    return {"L": L, "words": int(X.shape[0]),
            "sogrand": _bins(pred_s, miss_s, edges, min_count),
            "forney": _bins(pred_f, miss_f, edges, min_count),
            "overall": {"sogrand": (float(pred_s.sum()), int(miss_s.sum())),
                        "forney": (float(pred_f.sum()), int(miss_f.sum()))}}


def bit_probability_bins(code: Code, llr, X, L: int = 4, query_cap: int = 10**4, nbins: int = 20) -> list:
    """The paper's form of the bitwise check (Fig. BER_prediction): the
    predicted probability that a bit is 1, 1 / (1 + e^L_APP), in equal-width
    bins, against the frequency of 1 among the transmitted bits of each bin."""
    out = sogrand_decode(code, llr, L=L, query_cap=query_cap, lists=False)
    lapp = out["llr_app"].cpu().numpy().astype(np.float64)
    with np.errstate(over="ignore"):
        p1 = 1.0 / (1.0 + np.exp(lapp))
    ones = np.asarray(X, dtype=np.uint8) == 1
    edges = np.linspace(0.0, 1.0, nbins + 1)
    edges[-1] = 1.0 + 1e-12
    rows = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (p1 >= lo) & (p1 < hi)
        cnt = int(sel.sum())
        rows.append({"lo": float(lo), "hi": float(min(hi, 1.0)), "count": cnt,
                     "predicted": float(p1[sel].mean()) if cnt else None,
                     "empirical": float(ones[sel].mean()) if cnt else None})
    return rows


def bit_calibration(code: Code, llr, X, L: int = 4, query_cap: int = 10**4, forney: bool = False, edges=None,
                    min_count: int = 2000) -> list:
    """Binned predicted bit-error probability 1/(1+e^|L_APP|) vs the observed
    rate of hard-decision errors."""
    if edges is None:  # half-decade bins; the first also takes predictions of exactly 0 (infinite L_APP)
        edges = np.append(10.0 ** np.arange(-6.0, -0.5, 0.5), 0.5 + 1e-9)
        edges[0] = 0.0
    out = sogrand_decode(code, llr, L=L + (1 if forney else 0), query_cap=query_cap, lists=False, forney=forney)
    lapp = out["llr_app"].cpu().numpy().astype(np.float64)
    with np.errstate(over="ignore"):
        pred = 1.0 / (1.0 + np.exp(np.abs(lapp)))
    err = (lapp < 0).astype(np.uint8) != np.asarray(X, dtype=np.uint8)
    return _bins(pred.ravel(), err.ravel(), edges, min_count)
