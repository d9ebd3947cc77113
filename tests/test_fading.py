"""Pins of the block Rician fading / QPSK input generator (Sec. VI, Block
Fading Channels): fading statistics, the LLRs being log-likelihood ratios,
interleaving, and counter-based determinism."""
import numpy as np
import pytest

from workloads import ebch, fading_frames
from workloads.channel import sigma2_for


def test_fading_coefficients_are_rician_with_unit_power():
    code = ebch("ebch_32_26")
    K = 8.0
    _, _, _, H = fading_frames(code, 3000, 4.0, seed=5, Nc=256, t=2, K=K, return_h=True)
    assert H.shape == (3000, 2)
    assert abs((np.abs(H) ** 2).mean() - 1.0) < 0.02
    los = np.sqrt(K / (K + 1))
    assert abs(H.real.mean() - los) < 0.01 and abs(H.imag.mean()) < 0.01
    # scattered part: variance 1/(K+1) split over the two dimensions
    assert abs(H.real.var() - 0.5 / (K + 1)) < 0.01 and abs(H.imag.var() - 0.5 / (K + 1)) < 0.01


def test_llrs_are_log_likelihood_ratios_given_the_coefficient():
    """Given h, s * LLR (s = 1 - 2c) is Gaussian with mean 2|h|^2/sigma^2 and
    variance twice its mean: the consistency of a true LLR.  One coherence
    block per frame (t = 1, Nc = 512) so every frame has a single h."""
    code = ebch("ebch_32_26")
    F = 300
    ebn0 = 3.0
    U, X, L, H = fading_frames(code, F, ebn0, seed=6, Nc=512, t=1, K=2.0, return_h=True)
    s2 = float(sigma2_for(ebn0, code.k ** 2 / code.n ** 2))
    sl = (L.reshape(F, -1) * (1.0 - 2.0 * X.reshape(F, -1))).astype(np.float64)
    mu = 2.0 * np.abs(H[:, 0]) ** 2 / s2
    sel = mu > 1.0  # deep fades carry too little signal for a relative check
    np.testing.assert_allclose(sl[sel].mean(axis=1), mu[sel], rtol=0.1, atol=0.1)
    np.testing.assert_allclose(sl[sel].var(axis=1), 2.0 * mu[sel], rtol=0.25)
    # pooled over frames the relations hold tightly
    assert abs(sl.mean() / mu.mean() - 1.0) < 0.01
    assert abs((sl.var(axis=1).mean()) / (2.0 * mu.mean()) - 1.0) < 0.03


def test_interleaving_and_determinism():
    code = ebch("ebch_16_11")
    # n^2 = 256 = 2 t Nc
    U, X, L = fading_frames(code, 40, 30.0, seed=7, Nc=64, t=2, K=8)
    assert ((L < 0) == (X == 1)).mean() > 0.999  # high SNR: hard decisions are the codeword
    U2, X2, L2 = fading_frames(code, 10, 30.0, seed=7, Nc=64, t=2, K=8, first=17)
    np.testing.assert_array_equal(L2, L[17:27])
    np.testing.assert_array_equal(X2, X[17:27])
    with pytest.raises(ValueError):
        fading_frames(code, 1, 3.0, seed=1, Nc=100, t=2, K=8)
