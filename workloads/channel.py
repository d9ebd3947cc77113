"""Seeded BPSK-over-AWGN channel LLRs (input generation).

Convention (Sec. V-B): LLR = log p(r|0)/p(r|1); BPSK maps bit 0 -> +1 and bit 1
-> -1; with y = x + N(0, sigma^2) the channel LLR is L_Ch = 2y/sigma^2.  For a
code of rate R at a given Eb/N0, sigma^2 = 1 / (2 R Eb/N0).

Randomness is counter-based: frames are generated in fixed blocks of
``BLOCK`` frames, block b drawing from a Philox stream keyed by
SeedSequence([seed, stream, b]).  A frame's content therefore depends only on
(seed, stream, frame index), never on how a caller slices the range.
"""
from __future__ import annotations

import numpy as np

BLOCK = 256


def sigma2_for(ebn0_db, rate: float):
    return 1.0 / (2.0 * rate * np.power(10.0, np.asarray(ebn0_db, dtype=np.float64) / 10.0))


def _block_rng(seed: int, stream: int, block: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(stream), int(block)])))


def _frames_in_block(code, nbits_info, nbits, rate, ebn0_db, seed, stream, b, lo, hi, encode):
    rng = _block_rng(seed, stream, b)
    u = rng.integers(0, 2, size=(BLOCK, nbits_info), dtype=np.uint8)
    noise = rng.standard_normal(size=(BLOCK, nbits), dtype=np.float64)
    u = u[lo:hi]
    noise = noise[lo:hi]
    x = encode(u)
    s2 = sigma2_for(ebn0_db, rate)
    s2 = np.broadcast_to(np.asarray(s2, dtype=np.float64), (hi - lo,))[:, None]
    y = (1.0 - 2.0 * x.reshape(hi - lo, nbits).astype(np.float64)) + np.sqrt(s2) * noise
    llr = (2.0 * y / s2).astype(np.float32)
    return u, x, llr


def _generate(code, count, ebn0_db, seed, stream, first, nbits_info, nbits, rate, encode, threads=None):
    ebn0 = np.broadcast_to(np.asarray(ebn0_db, dtype=np.float64), (count,))
    jobs = []
    f = first
    end = first + count
    while f < end:
        b = f // BLOCK
        lo = f - b * BLOCK
        hi = min(BLOCK, end - b * BLOCK)
        jobs.append((b, lo, hi, f - first))
        f += hi - lo

    def run(job):
        b, lo, hi, o = job
        return _frames_in_block(code, nbits_info, nbits, rate, ebn0[o:o + hi - lo], seed, stream, b, lo, hi, encode)

    if threads and threads > 1 and len(jobs) > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(run, jobs))
    else:
        parts = [run(j) for j in jobs]
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
            np.concatenate([p[2] for p in parts]))


def awgn_frames(code, count: int, ebn0_db, seed: int, first: int = 0, stream: int = 1, threads: int | None = None,
                col_code=None, punctured=None):
    """Product-code frames: (U [F,k,k] u8, X [F,n,n] u8, L_Ch [F,n,n] f32).

    ``ebn0_db`` is a scalar or one value per frame; the rate is the product
    code's k^2/n^2.  With ``col_code`` the frames are of the product of the
    row code ``code`` and the column code: U [F,k_col,k_row], X and L_Ch
    [F,n_col,n_row], rate k_row k_col / (n_row n_col).  ``punctured`` (a 0/1
    mask of the frame's shape) marks coded bits that are not transmitted:
    their L_Ch is 0 (an erasure) and the rate counts only the sent bits.
    """
    r, c = code, (code if col_code is None else col_code)
    nbits = r.n * c.n
    sent = nbits if punctured is None else nbits - int(np.count_nonzero(punctured))
    if punctured is not None and np.shape(punctured) != (c.n, r.n):
        raise ValueError("punctured must have the frame's shape [n_col, n_row]")
    if col_code is None:
        n, k = code.n, code.k
        U, X, L = _generate(code, count, ebn0_db, seed, stream, first, k * k, nbits, (k * k) / sent,
                            lambda u: code.product_encode(u.reshape(-1, k, k)), threads)
    else:
        from .codes import product_encode
        U, X, L = _generate(code, count, ebn0_db, seed, stream, first, r.k * c.k, nbits, (r.k * c.k) / sent,
                            lambda u: product_encode(r, c, u.reshape(-1, c.k, r.k)), threads)
    L = L.reshape(-1, c.n, r.n)
    if punctured is not None:
        L[:, np.asarray(punctured, dtype=bool)] = 0.0
    return U.reshape(-1, c.k, r.k), X.reshape(-1, c.n, r.n), L


def awgn_words(code, count: int, ebn0_db, seed: int, first: int = 0, stream: int = 2, threads: int | None = None):
    """Independent component words: (U [W,k], X [W,n], L_Ch [W,n] f32) at the component rate."""
    return _generate(code, count, ebn0_db, seed, stream, first, code.k, code.n, code.k / code.n,
                     lambda u: code.encode(u), threads)
