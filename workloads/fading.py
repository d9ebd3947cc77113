"""Seeded block Rician fading with Gray-labelled QPSK (input generation).

The channel of the paper's fading experiments (Sec. VI, "Block Fading
Channels"): a frame of N coded bits is randomly interleaved, mapped two bits
per symbol to Gray-labelled QPSK x = Delta (s1 + j s2), s = 1 - 2c, and sent
over t coherence blocks of N_c symbols (N = 2 t N_c), each with its own fading
coefficient H = sqrt(K/(K+1)) + sqrt(1/(K+1)) H_Ra, H_Ra ~ CN(0, 1) (real and
imaginary parts of variance 1/2, so E|H|^2 = 1), and complex Gaussian noise
of variance sigma^2 per real dimension: y = H x + z.  With the coefficient
known at the receiver, the LLRs of the two bits of a symbol are
2 Delta Re(y h*) / sigma^2 and 2 Delta Im(y h*) / sigma^2; they are
de-interleaved back to codeword order.  Delta = 1, so Es/N0 = 1/sigma^2 and,
at rate R with two coded bits per symbol, sigma^2 = 1 / (2 R Eb/N0).

Randomness is counter-based as in ``channel``: block b of BLOCK frames draws
from SeedSequence([seed, stream, b]).
"""
from __future__ import annotations

import numpy as np

from .channel import BLOCK, _block_rng


def _fading_block(code, nbits_info, nbits, rate, ebn0_db, seed, stream, b, lo, hi, encode, Nc, t, K):
    rng = _block_rng(seed, stream, b)
    u = rng.integers(0, 2, size=(BLOCK, nbits_info), dtype=np.uint8)
    perm = np.argsort(rng.random(size=(BLOCK, nbits)), axis=1)       # interleaver of each frame
    hra = rng.standard_normal(size=(BLOCK, t, 2)) * np.sqrt(0.5)      # Rayleigh part, per coherence block
    z = rng.standard_normal(size=(BLOCK, t * Nc, 2))                   # unit-variance noise, scaled below
    u, perm, hra, z = u[lo:hi], perm[lo:hi], hra[lo:hi], z[lo:hi]
    x = encode(u).reshape(hi - lo, nbits)
    s2 = 1.0 / (2.0 * rate * np.power(10.0, np.asarray(ebn0_db, dtype=np.float64) / 10.0))
    s2 = np.broadcast_to(s2, (hi - lo,))[:, None]
    xi = np.take_along_axis(x, perm, axis=1).astype(np.float64)        # interleaved bits
    sym = (1.0 - 2.0 * xi[:, 0::2]) + 1j * (1.0 - 2.0 * xi[:, 1::2])   # Gray QPSK, Delta = 1
    h = np.sqrt(K / (K + 1.0)) + np.sqrt(1.0 / (K + 1.0)) * (hra[..., 0] + 1j * hra[..., 1])
    hs = np.repeat(h, Nc, axis=1)                                      # coefficient of every symbol
    y = hs * sym + np.sqrt(s2) * (z[..., 0] + 1j * z[..., 1])
    m = y * np.conj(hs)
    li = np.empty((hi - lo, nbits), dtype=np.float64)
    li[:, 0::2] = 2.0 * m.real / s2
    li[:, 1::2] = 2.0 * m.imag / s2
    llr = np.empty_like(li)
    np.put_along_axis(llr, perm, li, axis=1)                           # back to codeword order
    return u, x, llr.astype(np.float32), h


def fading_frames(code, count: int, ebn0_db, seed: int, Nc: int, t: int, K: float, first: int = 0, stream: int = 3,
                  threads: int | None = None, return_h: bool = False):
    """Product-code frames over block Rician fading with QPSK:
    (U [F,k,k] u8, X [F,n,n] u8, L_Ch [F,n,n] f32[, H [F,t] complex]).
    Requires n^2 = 2 t Nc."""
    n, k = code.n, code.k
    nbits, nbits_info, rate = n * n, k * k, (k * k) / (n * n)
    if 2 * t * Nc != nbits:
        raise ValueError(f"N = n^2 = {nbits} must equal 2 t Nc = {2 * t * Nc}")
    ebn0 = np.broadcast_to(np.asarray(ebn0_db, dtype=np.float64), (count,))
    encode = lambda u: code.product_encode(u.reshape(-1, k, k))  # noqa: E731
    jobs, f, end = [], first, first + count
    while f < end:
        b = f // BLOCK
        lo = f - b * BLOCK
        hi = min(BLOCK, end - b * BLOCK)
        jobs.append((b, lo, hi, f - first))
        f += hi - lo

    def run(job):
        b, lo, hi, o = job
        return _fading_block(code, nbits_info, nbits, rate, ebn0[o:o + hi - lo], seed, stream, b, lo, hi, encode,
                             Nc, t, K)

    if threads and threads > 1 and len(jobs) > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(run, jobs))
    else:
        parts = [run(j) for j in jobs]
    U = np.concatenate([p[0] for p in parts]).reshape(-1, k, k)
    X = np.concatenate([p[1] for p in parts]).reshape(-1, n, n)
    L = np.concatenate([p[2] for p in parts]).reshape(-1, n, n)
    if return_h:
        return U, X, L, np.concatenate([p[3] for p in parts])
    return U, X, L
