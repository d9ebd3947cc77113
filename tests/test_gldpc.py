"""Pins of the QC-GLDPC construction (Sec. VI, from Lentmaier et al.) and of
the oracle's QC-GLDPC decoder."""
import numpy as np

from workloads import ebch
from workloads.gldpc import QCGLDPC, diagonal_positions, gldpc_frames


def test_construction_follows_the_adjacency_matrix():
    n = 8
    pos = diagonal_positions(n)
    # second row of blocks: block column j is the identity rotated right by j,
    # so check d meets variable (block j, position (d + j) mod n)
    for d in range(n):
        for j in range(n):
            assert pos[d, j] == ((d + j) % n) * n + j
    g = QCGLDPC(ebch("ebch_16_11"))
    H, G = g.H.astype(np.int64), g.G.astype(np.int64)
    assert ((H @ G.T) % 2 == 0).all()
    # the dimension is n^2 - rank(H); the paper's nominal n^2 - 2n(n-k) counts every check as independent
    assert g.K >= 16 * 16 - 2 * 16 * 5
    assert np.linalg.matrix_rank(G.astype(float)) == g.K  # full-rank generator (over the reals, a necessary sign)
    # every row and every wrapped diagonal of a codeword is a component codeword
    c = ebch("ebch_32_26")
    g = QCGLDPC(c)
    U, X, L = gldpc_frames(g, 6, 3.0, seed=9)
    assert g.K == 646 and X.any()
    assert not c.syndrome(X.reshape(-1, 32)).any()
    assert not c.syndrome(X.reshape(6, -1)[:, diagonal_positions(32)].reshape(-1, 32)).any()


def test_oracle_gldpc_decoder(oracle_lib):
    c = ebch("ebch_32_26")
    g = QCGLDPC(c)
    oc = oracle_lib.OracleCode(c)
    U, X, L = gldpc_frames(g, 30, 2.5, seed=10)
    r = oracle_lib.gldpc_batch(oc, L, alpha=0.6, max_iter=20)
    dp = diagonal_positions(32)
    for f in range(30):
        B = r["bits"][f]
        ok = not c.syndrome(B).any() and not c.syndrome(B.reshape(-1)[dp]).any()
        assert ok == (r["status"][f] == 0)
    assert (r["status"] == 0).mean() > 0.8
    clean = (8.0 * (1.0 - 2.0 * X[:2])).astype(np.float32)
    r0 = oracle_lib.gldpc_batch(oc, clean)
    assert (r0["half_iters"] == 1).all() and (r0["bits"] == X[:2]).all()
    # not the product code: the same channel output decodes differently as a product frame
    rp = oracle_lib.product_batch(oc, L[:5], alpha=0.6, max_iter=20)
    assert (rp["half_iters"] != r["half_iters"][:5]).any() or (rp["bits"] != r["bits"][:5]).any()


def test_oracle_gldpc_fixes_weak_single_errors_in_the_first_half(oracle_lib):
    """One weak wrong-sign bit in every row of a clean frame: the row half
    corrects each row (its single flip is the first query of the right
    parity), so every row and wrapped diagonal is a codeword after one half."""
    c = ebch("ebch_32_26")
    g = QCGLDPC(c)
    oc = oracle_lib.OracleCode(c)
    U, X, L = gldpc_frames(g, 4, 3.0, seed=21)
    rng = np.random.default_rng(22)
    clean = (8.0 * (1.0 - 2.0 * X)).astype(np.float32)
    cols = rng.integers(0, 32, size=(4, 32))
    for f in range(4):
        clean[f, np.arange(32), cols[f]] *= -0.0625  # wrong sign, |LLR| = 0.5
    r = oracle_lib.gldpc_batch(oc, clean, alpha=0.6, max_iter=4)
    assert (r["half_iters"] == 1).all() and (r["status"] == 0).all()
    assert (r["bits"] == X).all()
