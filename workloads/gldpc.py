"""QC-GLDPC codes built on a short component code (input generation).

The (n^2, n^2 - 2n(n-k)) quasi-cyclic generalised LDPC code the paper takes
from Lentmaier et al. (Sec. VI): n^2 variable nodes in n blocks of n and two
rows of check nodes, each check a component codeword, with adjacency blocks
I^(0) ... I^(0) in the first row and I^(0), I^(1), ..., I^(n-1) in the second
(I^(s): the identity rotated right by s).  Writing the variables as an n x n
array X[r][j] (block j, position r), the first row of checks makes every row
r of X a component word (bit j = X[r][j]) and the second every wrapped
diagonal d (bit j = X[(d + j) mod n][j]).  A product code is the same
construction with columns in place of diagonals.

The generator is a basis of the null space of the full parity-check matrix
over GF(2), of dimension n^2 minus its rank.  The checks are not all
independent: for the eBCH components used here the rank falls n - k short of
2n(n-k) (eBCH(32,26): rank 378, K = 646 against the nominal 640).
"""
from __future__ import annotations

import numpy as np

from .codes import LinearCode


def diagonal_positions(n: int) -> np.ndarray:
    """[n, n]: flat index r * n + j of bit j of wrapped diagonal d (row (d + j) mod n)."""
    d = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return ((d + j) % n) * n + j


def _gf2_nullspace(H: np.ndarray) -> np.ndarray:
    """Basis (rows) of {x : H x = 0 over GF(2)} by elimination on 64-bit packed rows."""
    m, N = H.shape
    W = (N + 63) // 64
    bits = np.zeros((m, W * 64), np.uint8)
    bits[:, :N] = H
    M = np.packbits(bits.reshape(m, W, 64)[:, :, ::-1], axis=2, bitorder="big").view(">u8").reshape(m, W)
    M = M.astype(np.uint64)
    pivots = []
    row = 0
    for c in range(N):
        if row == m:
            break
        w, b = c >> 6, np.uint64(c & 63)
        col = (M[row:, w] >> b) & np.uint64(1)
        nz = np.nonzero(col)[0]
        if nz.size == 0:
            continue
        p = row + nz[0]
        if p != row:
            M[[row, p]] = M[[p, row]]
        hit = ((M[:, w] >> b) & np.uint64(1)).astype(bool)
        hit[row] = False
        M[hit] ^= M[row]
        pivots.append(c)
        row += 1
    R = np.unpackbits(M.astype(">u8").view(np.uint8).reshape(m, W, 8), axis=2, bitorder="big")
    R = R.reshape(m, W, 64)[:, :, ::-1].reshape(m, W * 64)[:row, :N]
    free = np.setdiff1d(np.arange(N), np.array(pivots, dtype=np.int64))
    G = np.zeros((free.size, N), np.uint8)
    G[np.arange(free.size), free] = 1
    G[:, pivots] = R[:, free].T
    return G


class QCGLDPC:
    """QC-GLDPC code of a component code: rows and wrapped diagonals of an n x n array."""

    def __init__(self, comp: LinearCode):
        self.comp = comp
        n, m = comp.n, comp.n - comp.k
        self.n_comp = n
        self.N = n * n
        rows = np.arange(n * n).reshape(n, n)
        diags = diagonal_positions(n)
        H = np.zeros((2 * n * m, n * n), np.uint8)
        for s, pos in enumerate((rows, diags)):
            for w in range(n):
                H[(s * n + w) * m:(s * n + w + 1) * m][:, pos[w]] = comp.H
        self.H = H
        self.G = _gf2_nullspace(H)
        self.K = self.G.shape[0]

    def encode(self, U: np.ndarray) -> np.ndarray:
        """[F, K] information bits -> [F, n, n] codewords (X[r][j])."""
        U = np.asarray(U, dtype=np.uint8)
        X = (U.astype(np.int64) @ self.G.astype(np.int64)) & 1
        return X.astype(np.uint8).reshape(-1, self.n_comp, self.n_comp)


def gldpc_frames(code: QCGLDPC, count: int, ebn0_db, seed: int, first: int = 0, stream: int = 4,
                 threads: int | None = None):
    """Codeword frames over BPSK/AWGN: (U [F,K], X [F,n,n], L_Ch [F,n,n] f32), rate K/n^2."""
    from .channel import _generate
    n = code.n_comp
    U, X, L = _generate(code, count, ebn0_db, seed, stream, first, code.K, n * n, code.K / (n * n),
                        lambda u: code.encode(u), threads)
    return U, X.reshape(-1, n, n), L.reshape(-1, n, n)
