"""Even linear component codes and the product-code encoder (input generation).

The paper decodes product codes whose component codes are *even* linear block
codes (Sec. III-B): every codeword has even weight, so the parity of the
demodulated word equals the parity of the noise.  A non-even code is made even
by appending an overall parity bit, G_{i,n+1} = sum_j G_{i,j} (Sec. III-B).

The component codes here are extended BCH codes: a binary primitive BCH code of
length 2^m - 1 (generator = lcm of the minimal polynomials of alpha^1, alpha^3,
..., alpha^(2t-1)) followed by the overall-parity extension.  t = 1 gives the
extended Hamming codes.

Bit layout of a component codeword (length n = 2^m):
    positions 0 .. k-1        information bits u_0 .. u_{k-1}
    positions k .. n-2        remainder of x^(n0-k) u(x) mod g(x) (n0 = n-1)
    position  n-1             overall parity
Product codes (Sec. VI, Elias): a k x k information block is encoded row by
row, then every one of the n columns is encoded; the frame is the n x n matrix
in row-major order (bit (i, j) at index i*n + j).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# name -> (n, k, m, primitive polynomial as int (bit i = coeff of x^i), t)
CODE_SPECS = {
    "ebch_8_4": (8, 4, 3, 0b1011, 1),            # x^3+x+1
    "ebch_16_11": (16, 11, 4, 0b10011, 1),       # x^4+x+1
    "ebch_16_7": (16, 7, 4, 0b10011, 2),
    "ebch_32_26": (32, 26, 5, 0b100101, 1),      # x^5+x^2+1
    "ebch_64_57": (64, 57, 6, 0b1000011, 1),     # x^6+x+1
    "ebch_64_51": (64, 51, 6, 0b1000011, 2),     # g = m1*m3 over GF(64)
    "ebch_128_120": (128, 120, 7, 0b10001001, 1),  # x^7+x^3+1
}


def _gf_tables(m: int, prim: int):
    q = 1 << m
    exp = np.zeros(2 * q, dtype=np.int64)
    log = np.full(q, -1, dtype=np.int64)
    x = 1
    for i in range(q - 1):
        exp[i] = x
        log[x] = i
        x <<= 1
        if x & q:
            x ^= prim
    if x != 1:
        raise ValueError("polynomial is not primitive")
    for i in range(q - 1, 2 * q):
        exp[i] = exp[i - (q - 1)]
    return exp, log


def _minimal_polynomial(m: int, prim: int, e: int) -> list[int]:
    """Coefficients (low degree first, over GF(2)) of the minimal polynomial of alpha^e."""
    exp, log = _gf_tables(m, prim)
    order = (1 << m) - 1
    coset = []
    x = e % order
    while x not in coset:
        coset.append(x)
        x = (2 * x) % order
    poly = [1]  # GF(2^m) elements
    for root_e in coset:
        root = exp[root_e]
        nxt = [0] * (len(poly) + 1)
        for i, a in enumerate(poly):
            nxt[i + 1] ^= a  # a * x
            if a:
                nxt[i] ^= exp[log[a] + log[root]]  # a * root
        poly = nxt
    if any(c not in (0, 1) for c in poly):
        raise AssertionError("minimal polynomial not binary")
    return [int(c) for c in poly]


def _polymul2(a: list[int], b: list[int]) -> list[int]:
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] ^= y
    return out


def bch_generator(m: int, prim: int, t: int) -> list[int]:
    """Generator polynomial of the primitive narrow-sense BCH code of length 2^m-1."""
    order = (1 << m) - 1
    seen: set[int] = set()
    g = [1]
    for i in range(1, 2 * t, 2):
        e = i % order
        coset = set()
        x = e
        while x not in coset:
            coset.add(x)
            x = (2 * x) % order
        if coset & seen:
            continue
        seen |= coset
        g = _polymul2(g, _minimal_polynomial(m, prim, e))
    return g


def _systematic_generator(n0: int, g: list[int]) -> np.ndarray:
    """k x n0 matrix [I_k | P]; row i encodes the unit message e_i."""
    r = len(g) - 1
    k = n0 - r
    G = np.zeros((k, n0), dtype=np.uint8)
    for i in range(k):
        # remainder of x^(r+i) mod g(x)
        rem = [0] * (r + i) + [1]
        for d in range(len(rem) - 1, r - 1, -1):
            if rem[d]:
                for j, gj in enumerate(g):
                    rem[d - r + j] ^= gj
        G[i, i] = 1
        G[i, k:] = np.array(rem[:r], dtype=np.uint8)
    return G


@dataclass
class LinearCode:
    """A binary linear code given by G (k x n) and H ((n-k) x n), entries 0/1."""

    name: str
    n: int
    k: int
    G: np.ndarray
    H: np.ndarray
    even: bool = field(default=True)

    @property
    def rate(self) -> float:
        return self.k / self.n

    def encode(self, u: np.ndarray) -> np.ndarray:
        """Encode rows of u ([..., k] uint8) into [..., n] uint8."""
        u = np.asarray(u, dtype=np.uint8)
        out = (u.astype(np.float32) @ self.G.astype(np.float32)).astype(np.int64) & 1
        return out.astype(np.uint8)

    def syndrome(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.uint8)
        return ((x.astype(np.float32) @ self.H.T.astype(np.float32)).astype(np.int64) & 1).astype(np.uint8)

    def product_encode(self, U: np.ndarray) -> np.ndarray:
        """[F, k, k] information blocks -> [F, n, n] product codewords (rows first, then columns)."""
        U = np.asarray(U, dtype=np.uint8)
        F = U.shape[0]
        rows = self.encode(U.reshape(F * self.k, self.k)).reshape(F, self.k, self.n)
        cols = self.encode(np.ascontiguousarray(rows.transpose(0, 2, 1)).reshape(F * self.n, self.k))
        return np.ascontiguousarray(cols.reshape(F, self.n, self.n).transpose(0, 2, 1))


def product_encode(row: LinearCode, col: LinearCode, U: np.ndarray) -> np.ndarray:
    """[F, k_col, k_row] information blocks -> [F, n_col, n_row] product
    codewords of the row and column codes (rows first, then columns): every
    row is a row-code word, every column a column-code word."""
    U = np.asarray(U, dtype=np.uint8)
    F = U.shape[0]
    rows = row.encode(U.reshape(F * col.k, row.k)).reshape(F, col.k, row.n)
    cols = col.encode(np.ascontiguousarray(rows.transpose(0, 2, 1)).reshape(F * row.n, col.k))
    return np.ascontiguousarray(cols.reshape(F, row.n, col.n).transpose(0, 2, 1))


def shorten(code: LinearCode, s: int) -> LinearCode:
    """The (n - s, k - s) code of `code` (systematic, G = [I_k | P]) shortened
    by its first s information positions: codewords of `code` that are zero
    there, with those positions deleted (G' = G[s:, s:], H' = H[:, s:]).  An
    even code stays even (its all-ones check restricted to the kept positions).
    Rate adaptation of product codes by shortening (Sec. VII) uses such
    components."""
    if not 0 <= s < code.k:
        raise ValueError("0 <= s < k")
    if not (code.G[:, :code.k] == np.eye(code.k, dtype=np.uint8)).all():
        raise ValueError("shortening needs a systematic generator [I_k | P]")
    return LinearCode(name=f"{code.name}_s{s}", n=code.n - s, k=code.k - s,
                      G=np.ascontiguousarray(code.G[s:, s:]), H=np.ascontiguousarray(code.H[:, s:]), even=code.even)


def ebch(name_or_nk) -> LinearCode:
    """Extended BCH code by name ('ebch_64_57') or by (n, k)."""
    if isinstance(name_or_nk, tuple):
        name = f"ebch_{name_or_nk[0]}_{name_or_nk[1]}"
    else:
        name = name_or_nk
    n, k, m, prim, t = CODE_SPECS[name]
    n0 = n - 1
    g = bch_generator(m, prim, t)
    G0 = _systematic_generator(n0, g)
    if G0.shape[0] != k:
        raise AssertionError(f"{name}: dimension {G0.shape[0]} != {k}")
    par = (G0.sum(axis=1) & 1).astype(np.uint8)[:, None]
    G = np.concatenate([G0, par], axis=1)
    P = G0[:, k:]  # k x (n0-k)
    r = n0 - k
    H0 = np.concatenate([P.T, np.eye(r, dtype=np.uint8), np.zeros((r, 1), dtype=np.uint8)], axis=1)
    H = np.concatenate([H0, np.ones((1, n), dtype=np.uint8)], axis=0)
    return LinearCode(name=name, n=n, k=k, G=G, H=H.astype(np.uint8), even=True)
