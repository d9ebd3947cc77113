"""Pins of the oracle's 1-line ORBGRAND query order and its parameter c.

The paper takes the order from the 1-line ORBGRAND variant (Sec. III-B and
VI cite it), generated by the landslide algorithm as integer partitions into
distinct parts.  Pins, none of which re-uses the oracle's generator:
* per (cost, Hamming weight) group, the number of patterns equals the number
  of partitions of cost - c*w into w distinct parts <= n (textbook
  recurrence);
* the whole class is covered, every pattern exactly once (n = 12);
* cost is nondecreasing; ties by weight, then lexicographic rank vectors;
* the even-code parity skip only emits weights of the class parity;
* c equals an exact rational least-squares recomputation, and a perfectly
  linear reliability profile beta*(r + c0) returns c0.
"""
from fractions import Fraction
from functools import lru_cache
import math

import numpy as np
import pytest


@lru_cache(maxsize=None)
def distinct_partitions(m, w, n):
    """# of partitions of m into exactly w distinct parts, each <= n."""
    if w == 0:
        return 1 if m == 0 else 0
    if n <= 0 or m <= 0:
        return 0
    return distinct_partitions(m, w, n - 1) + distinct_partitions(m - n, w - 1, n - 1)


@pytest.mark.parametrize("n,c,cls", [(8, 0, -1), (16, 0, 0), (16, 2, 1), (32, 1, 0), (32, 5, 1), (64, 3, 0),
                                     (64, 0, 1), (64, 20, 0), (128, 4, 0)])
def test_group_counts_are_distinct_partition_counts(oracle_lib, n, c, cls):
    ranks, cost, w = oracle_lib.trace(n, c, cls, 4000)
    assert (np.diff(cost) >= 0).all()
    pos = np.arange(1, n + 1)
    assert (ranks.sum(axis=1) == w).all()
    assert ((ranks * pos).sum(axis=1) + c * w == cost).all()
    if cls >= 0:
        assert ((w & 1) == cls).all()
    last = cost[-1]
    groups = {}
    for cc, ww in zip(cost.tolist(), w.tolist()):
        groups[(cc, ww)] = groups.get((cc, ww), 0) + 1
    # every complete level: all groups present with the partition counts
    for C in range(0, last):
        for ww in range(0, n + 1):
            if cls >= 0 and (ww & 1) != cls:
                continue
            m = C - c * ww
            expect = distinct_partitions(m, ww, n) if m >= 0 else 0
            assert groups.get((C, ww), 0) == expect, (C, ww)


@pytest.mark.parametrize("n,c,cls", [(16, 0, 0), (16, 3, 1), (64, 2, 0)])
def test_tie_order_weight_then_lexicographic(oracle_lib, n, c, cls):
    ranks, cost, w = oracle_lib.trace(n, c, cls, 3000)
    vecs = [tuple(np.nonzero(r)[0] + 1) for r in ranks]
    for a in range(len(vecs) - 1):
        ka = (int(cost[a]), int(w[a]), vecs[a])
        kb = (int(cost[a + 1]), int(w[a + 1]), vecs[a + 1])
        assert ka < kb


@pytest.mark.parametrize("cls,c", [(-1, 0), (0, 0), (1, 0), (0, 3), (1, 7)])
def test_full_coverage_each_pattern_once(oracle_lib, cls, c):
    n = 12
    total = 2 ** n if cls < 0 else 2 ** (n - 1)
    ranks, cost, w = oracle_lib.trace(n, c, cls, total + 10)
    assert ranks.shape[0] == total
    keys = ranks.astype(np.int64) @ (1 << np.arange(n, dtype=np.int64))
    assert len(np.unique(keys)) == total
    pop = np.array([bin(int(k)).count("1") for k in keys])
    if cls >= 0:
        assert ((pop & 1) == cls).all()


def _c_exact(absl_sorted, c_max):
    n = len(absl_sorted)
    amax = (1 << 20) - 1
    a = []
    for v in absl_sorted:
        fv = Fraction(float(np.float32(v)))
        a.append(min(amax, math.floor(fv * 256 + Fraction(1, 2))))
    r = list(range(1, n + 1))
    mr = Fraction(sum(r), n)
    ma = Fraction(sum(a), n)
    sxy = sum((ri - mr) * (ai - ma) for ri, ai in zip(r, a))
    sxx = sum((ri - mr) ** 2 for ri in r)
    beta = sxy / sxx
    if beta <= 0:
        return 0
    b = ma - beta * mr
    c = math.floor(b / beta + Fraction(1, 2))
    return max(0, min(c_max, c))


def test_one_line_c_matches_exact_least_squares(oracle_lib):
    rng = np.random.default_rng(5)
    for trial in range(300):
        n = [8, 16, 32, 64, 128][trial % 5]
        scale = [0.5, 3.0, 20.0, 300.0, 5000.0][trial % 5]
        v = np.sort(np.abs(rng.normal(1.0, 1.0, n) * scale)).astype(np.float32)
        if trial % 7 == 0:
            v[: n // 4] = 0.0
        assert oracle_lib.one_line_c(v, n) == _c_exact(v, n)


def test_one_line_c_linear_profile_and_limits(oracle_lib):
    for n in (16, 64, 128):
        for s in (1, 3, 17):
            for c0 in (0, 1, 4, 9):
                a = s * (np.arange(1, n + 1) + c0)
                v = (a / 256.0).astype(np.float32)
                assert oracle_lib.one_line_c(v, n) == min(c0, n)
        v = np.full(n, 2.5, np.float32)  # flat: slope 0 -> c = 0
        assert oracle_lib.one_line_c(v, n) == 0
        v = (np.arange(1, n + 1) * 0.001 + 50).astype(np.float32)  # very flat, big intercept -> clamp
        assert oracle_lib.one_line_c(v, n) == n
