"""The QCrank read-out of the oracle against its pins (CPU only).

Pins: a hand-counted set of shots (address and data bits, the 2/pi arcsin
sqrt inverse, an address without shots), the inverse of the closed form
P(1 | j) = sin^2(pi pixel / 2) with exact probabilities, and the shot-noise
law of the estimate: by the delta method the pixel error has variance
1 / (pi^2 s) with s shots per address (Table 2: s = 3000)."""
import numpy as np
import pytest

import oracle
from oracle import qcrank_ref as Q
import workloads as W


def test_hand_counted_shots():
    # a = 1 (bit 0), d = 2 (bits 1, 2)
    shots = [0b000, 0b010, 0b011, 0b111, 0b101]
    pix, counts, ones = Q.decode(shots, 1, 2)
    assert counts.tolist() == [2, 3]
    assert ones.tolist() == [[1, 0], [2, 2]]
    assert pix[0, 0] == pytest.approx(0.5, abs=1e-15)  # (2/pi) asin(sqrt(1/2))
    assert pix[0, 1] == 0.0
    assert pix[1, 0] == pytest.approx(2 / np.pi * np.arcsin(np.sqrt(2 / 3)), abs=1e-15)
    assert pix[1, 1] == pix[1, 0]
    # address 1 of a = 2 draws nothing
    pix2, counts2, _ = Q.decode([0b0100, 0b0000, 0b1110], 2, 2)
    assert counts2.tolist() == [2, 0, 1, 0]
    assert np.isnan(pix2[1]).all() and np.isnan(pix2[3]).all()
    assert np.abs(pix2[0] - [0.5, 0.0]).max() < 1e-15 and np.abs(pix2[2] - 1.0).max() < 1e-15


def test_exact_probabilities_invert_the_encoding():
    rng = np.random.default_rng(3)
    a, d = 5, 4
    pix = rng.uniform(0, 1, size=(1 << a, d))
    # the closed-form distribution, written out directly
    th = np.pi * pix
    amp = np.full((1 << d, 1 << a), 2.0 ** (-a / 2))
    for k in range(d):
        y = (np.arange(1 << d) >> k) & 1
        amp *= np.where(y[:, None] == 1, np.sin(th[:, k] / 2), np.cos(th[:, k] / 2))
    got = Q.pixels_from_probs(amp.reshape(-1) ** 2, a, d)
    assert np.abs(got - pix).max() < 1e-12
    # and the oracle's own simulation of the generated circuit
    psi = oracle.apply_circuit(a + d, W.qcrank(a, d, pix))
    got = Q.pixels_from_probs(oracle.probs(psi), a, d)
    assert np.abs(got - pix).max() < 1e-11
    assert Q.correlation(got, pix) > 1 - 1e-12


def test_shot_noise_law():
    """s shots per address: mean squared pixel error ~ 1 / (pi^2 s)."""
    a, d, s = 8, 6, 3000
    rng = np.random.default_rng(11)
    pix = rng.uniform(0.1, 0.9, size=(1 << a, d))  # away from the ends, where the delta method holds
    psi = oracle.apply_circuit(a + d, W.qcrank(a, d, pix))
    u = oracle.uniforms(5, s << a)
    shots = oracle.sample(psi, u)
    est, counts, _ = Q.decode(shots, a, d)
    assert counts.sum() == s << a
    mse = np.mean((est - pix) ** 2)
    want = 1.0 / (np.pi ** 2 * s)
    assert 0.8 * want < mse < 1.2 * want, (mse, want)
    assert Q.correlation(est, pix) > 0.999
