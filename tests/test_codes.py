"""Pins of the input generators: component codes, product encoder, channel.

The codes are inputs of the method (the paper's eBCH components, Sec. III-B
and VI), so they are pinned against textbook facts that do not come from the
construction itself: H G^T = 0, evenness, the weight-4 count of extended
Hamming codes A_4 = n(n-1)(n-2)/24, and the minimum distance 6 of eBCH(64,51).
"""
import itertools

import numpy as np
import pytest

from workloads import CODE_SPECS, awgn_frames, awgn_words, ebch, sigma2_for


@pytest.mark.parametrize("name", sorted(CODE_SPECS))
def test_generator_parity_check_orthogonal_and_even(name):
    c = ebch(name)
    assert c.G.shape == (c.k, c.n) and c.H.shape == (c.n - c.k, c.n)
    assert not ((c.G.astype(int) @ c.H.T.astype(int)) % 2).any()
    # systematic: information bits first
    assert (c.G[:, :c.k] == np.eye(c.k, dtype=np.uint8)).all()
    # even code: every generator row (hence every codeword) has even weight
    assert not (c.G.sum(axis=1) % 2).any()
    # full rank H over GF(2)
    M = c.H.copy().astype(np.uint8)
    rank = 0
    for col in range(c.n):
        piv = [r for r in range(rank, M.shape[0]) if M[r, col]]
        if not piv:
            continue
        M[[rank, piv[0]]] = M[[piv[0], rank]]
        for r in range(M.shape[0]):
            if r != rank and M[r, col]:
                M[r] ^= M[rank]
        rank += 1
    assert rank == c.n - c.k


def _count_zero_xor_subsets(H, w):
    cols = [int("".join(map(str, H[:, i])), 2) for i in range(H.shape[1])]
    n = len(cols)
    if w == 4:
        # pairs-of-pairs: count 4-subsets whose columns XOR to zero
        from collections import defaultdict
        pairs = defaultdict(list)
        for i in range(n):
            for j in range(i + 1, n):
                pairs[cols[i] ^ cols[j]].append((i, j))
        cnt = 0
        for lst in pairs.values():
            for (a, b), (c_, d) in itertools.combinations(lst, 2):
                if len({a, b, c_, d}) == 4:
                    cnt += 1
        return cnt // 3  # each 4-set is split into two pairs in 3 ways
    return sum(1 for s in itertools.combinations(cols, w) if np.bitwise_xor.reduce(s) == 0)


@pytest.mark.parametrize("name", ["ebch_8_4", "ebch_16_11", "ebch_32_26", "ebch_64_57"])
def test_extended_hamming_weight4_count(name):
    c = ebch(name)
    n = c.n
    assert _count_zero_xor_subsets(c.H, 4) == n * (n - 1) * (n - 2) // 24
    # minimum distance 4: no 1, 2 or 3 columns XOR to zero
    assert all(_count_zero_xor_subsets(c.H, w) == 0 for w in (1, 2, 3))


def test_ebch_64_51_minimum_distance_6():
    c = ebch("ebch_64_51")
    cols = np.array([int("".join(map(str, c.H[:, i])), 2) for i in range(c.n)], dtype=np.int64)
    assert len(set(cols.tolist())) == c.n and 0 not in cols  # d > 2
    # d > 4 (so d >= 6 for an even code): no two distinct pairs share an XOR
    seen = {}
    for i in range(c.n):
        for j in range(i + 1, c.n):
            x = int(cols[i] ^ cols[j])
            assert x not in seen, "four columns XOR to zero"
            seen[x] = (i, j)
    # d = 6 is attained: some 6 columns XOR to zero (search triples)
    triples = {}
    found = False
    for a, b, d in itertools.combinations(range(c.n), 3):
        x = int(cols[a] ^ cols[b] ^ cols[d])
        if x in triples and not ({a, b, d} & set(triples[x])):
            found = True
            break
        triples.setdefault(x, (a, b, d))
    assert found


def test_product_encoder_rows_and_columns_are_codewords():
    c = ebch("ebch_16_11")
    rng = np.random.default_rng(0)
    U = rng.integers(0, 2, size=(7, c.k, c.k), dtype=np.uint8)
    X = c.product_encode(U)
    assert (X[:, :c.k, :c.k] == U).all()
    for f in range(7):
        assert not c.syndrome(X[f]).any()
        assert not c.syndrome(X[f].T).any()


def test_channel_llr_statistics_and_determinism():
    c = ebch("ebch_32_26")
    U, X, L = awgn_frames(c, 300, 3.0, seed=11)
    U2, X2, L2 = awgn_frames(c, 40, 3.0, seed=11, first=260)
    assert np.array_equal(L[260:], L2) and np.array_equal(X[260:], X2)
    s2 = sigma2_for(3.0, (26 * 26) / (32 * 32))
    # LLR = 2y/s2 with y ~ N(1 - 2x, s2): mean 2/s2 (sign by bit), variance 4/s2
    sgn = 1.0 - 2.0 * X.astype(np.float64)
    z = L.astype(np.float64) * sgn
    assert abs(z.mean() - 2 / s2) < 0.02 * (2 / s2)
    assert abs(z.var() - 4 / s2) < 0.03 * (4 / s2)
    _, Xw, Lw = awgn_words(c, 1000, [2.0, 5.0] * 500, seed=3)
    err = ((Lw < 0) != Xw).mean(axis=1)
    assert err[0::2].mean() > 2 * err[1::2].mean()
