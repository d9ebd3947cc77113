"""Rate adaptation of product codes (Sec. VII): shortened component codes
and punctured frames, as input generators and through the oracle."""
import math

import numpy as np

from workloads import awgn_frames, ebch, shorten


def test_shortened_codes():
    rng = np.random.default_rng(4)
    for nm, s in [("ebch_16_11", 3), ("ebch_32_26", 6), ("ebch_64_57", 4)]:
        c = ebch(nm)
        sc = shorten(c, s)
        assert (sc.n, sc.k, sc.even) == (c.n - s, c.k - s, True)
        assert not ((sc.H.astype(np.int64) @ sc.G.T.astype(np.int64)) % 2).any()
        assert np.linalg.matrix_rank(sc.G.astype(float)) == sc.k
        U = rng.integers(0, 2, (64, sc.k), dtype=np.uint8)
        X = sc.encode(U)
        # a shortened codeword with the s deleted zeros put back is a codeword of the mother code
        assert not c.syndrome(np.concatenate([np.zeros((64, s), np.uint8), X], axis=1)).any()
        assert (X.sum(axis=1) % 2 == 0).all()
        assert (X[:, :sc.k] == U).all()  # still systematic
    # (13, 8) from eBCH(16,11): minimum distance 4, as the mother code's (brute force over 2^8 words)
    sc = shorten(ebch("ebch_16_11"), 3)
    U = ((np.arange(1, 256)[:, None] >> np.arange(8)) & 1).astype(np.uint8)
    assert sc.encode(U).sum(axis=1).min() == 4


def _permutation_mask(n, shift):
    m = np.zeros((n, n), bool)
    m[np.arange(n), (np.arange(n) * shift + 3) % n] = True
    return m


def test_punctured_frames_are_erasures_at_the_sent_rate():
    code = ebch("ebch_32_26")
    mask = _permutation_mask(32, 7)
    U, X, L = awgn_frames(code, 20, 3.0, seed=5, punctured=mask)
    # the same noise draws, unpunctured, at the Eb/N0 of the rate over all n^2 bits
    U2, X2, L2 = awgn_frames(code, 20, 3.0 + 10 * math.log10(1024 / (1024 - 32)), seed=5)
    assert (U == U2).all() and (X == X2).all()
    assert (L[:, mask] == 0).all() and (L[:, ~mask] != 0).all()
    np.testing.assert_allclose(L[:, ~mask], L2[:, ~mask], rtol=1e-6)


def test_oracle_fills_one_erasure_per_row_and_decodes_shortened_frames(oracle_lib):
    code = ebch("ebch_32_26")
    mask = _permutation_mask(32, 5)
    U, X, L = awgn_frames(code, 6, 3.0, seed=6, punctured=mask)
    clean = (8.0 * (1.0 - 2.0 * X)).astype(np.float32)
    clean[:, mask] = 0.0
    assert (X[:, mask] == 1).any()  # some erased bits are ones: the hard decision 0 is wrong there
    r = oracle_lib.product_batch(oracle_lib.OracleCode(code), clean, L=4, alpha=0.5, max_iter=4)
    assert (r["half_iters"] == 1).all() and (r["status"] == 0).all() and (r["bits"] == X).all()
    sc = shorten(ebch("ebch_64_57"), 4)
    U, X, L = awgn_frames(sc, 3, 3.0, seed=7)
    assert X.shape == (3, 60, 60)
    clean = (8.0 * (1.0 - 2.0 * X)).astype(np.float32)
    r = oracle_lib.product_batch(oracle_lib.OracleCode(sc), clean, L=4, alpha=0.5, max_iter=4)
    assert (r["half_iters"] == 1).all() and (r["bits"] == X).all()
