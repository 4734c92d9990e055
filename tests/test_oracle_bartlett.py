"""Pins of the dense Bartlett oracle (Appendix A, Algorithm 2 with one segment).

Each pin checks the oracle against the mathematics, not against itself: a dense DFT
written out as a matrix product, the exponential law of the H0 bin power (mean
sigma_n^2 ||w||^2, Appendix A), the Swerling-I detection probability that law implies,
and exact recovery of noise-free on-grid tones.
"""
import math

import numpy as np
import pytest
from scipy.stats import beta as beta_dist

import oracle as O
import rsft_inputs as ri


def _cp(hits, total, alpha=0.001):
    lo = beta_dist.ppf(alpha / 2, hits, total - hits + 1) if hits > 0 else 0.0
    hi = beta_dist.ppf(1 - alpha / 2, hits + 1, total - hits) if hits < total else 1.0
    return lo, hi


def test_spectrum_is_the_windowed_dense_dft():
    rng = np.random.default_rng(5)
    n = (8, 16)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    out = O.bartlett(x, "cheb", 40.0, 1.0, 1e-3)
    w0, w1 = O.bartlett_window(n, "cheb", 40.0)
    f0 = np.exp(-2j * np.pi * np.outer(np.arange(8), np.arange(8)) / 8)
    f1 = np.exp(-2j * np.pi * np.outer(np.arange(16), np.arange(16)) / 16)
    dense = f0 @ (np.outer(w0, w1) * x) @ f1.T
    np.testing.assert_allclose(out["spectrum"], dense, rtol=0, atol=1e-10)


def test_noise_only_power_is_exponential_and_pfa_holds():
    n, nv, p_fa = (64, 64), 3.0, 0.01
    ratios, hits, total = [], 0, 0
    for frame in range(12):
        x = ri.tone_cube(n, None, nv, 7000 + frame).astype(np.complex128)
        out = O.bartlett(x, "cheb", 60.0, nv, p_fa)
        energy = math.prod(float(np.sum(w ** 2)) for w in out["windows"])
        ratios.append(out["power"].reshape(-1) / (nv * energy))
        hits += len(out["located"])
        total += out["power"].size
    r = np.concatenate(ratios)
    se = 1.0 / math.sqrt(len(r))
    assert abs(r.mean() - 1.0) < 6 * se
    assert abs(np.mean(r > math.log(2)) - 0.5) < 6 * 0.5 * se
    lo, hi = _cp(hits, total)
    assert lo <= p_fa <= hi


def test_swerling1_detection_probability():
    # a Rayleigh-amplitude on-grid tone: the bin power is exponential with mean
    # sigma_b^2 |sum w|^2 + sigma_n^2 ||w||^2, so Pd = Pfa^(1 / (1 + SNR alpha'/beta'))
    n, nv, p_fa, sigma_b2 = (16, 16), 1.0, 1e-3, 0.05
    rng = np.random.default_rng(11)
    ws = O.bartlett_window(n, "cheb", 50.0)
    alpha = math.prod(float(np.sum(w)) ** 2 for w in ws)
    beta = math.prod(float(np.sum(w ** 2)) for w in ws)
    snr_gain = sigma_b2 * alpha / (nv * beta)
    pd = O.bartlett_pd_swerling1(p_fa, snr_gain)
    assert 0.2 < pd < 0.8
    k = (3, 9)
    t0, t1 = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    tone = np.exp(2j * np.pi * (k[0] * t0 + k[1] * t1) / 16)
    trials, hits = 3000, 0
    for _ in range(trials):
        a = (rng.standard_normal() + 1j * rng.standard_normal()) * math.sqrt(sigma_b2 / 2)
        noise = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * math.sqrt(nv / 2)
        out = O.bartlett(a * tone + noise, "cheb", 50.0, nv, p_fa)
        hits += int(np.ravel_multi_index(k, n) in set(out["located"].tolist()))
    lo, hi = _cp(hits, trials)
    assert lo <= pd <= hi


def test_exact_recovery_of_on_grid_tones():
    n = (32, 64)
    rng = np.random.default_rng(2)
    bins = [(1, 5), (7, 60), (30, 33)]
    amps = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    t0, t1 = np.meshgrid(np.arange(32), np.arange(64), indexing="ij")
    x = sum(a * np.exp(2j * np.pi * (k0 * t0 / 32 + k1 * t1 / 64)) for a, (k0, k1) in zip(amps, bins))
    out = O.bartlett(x, "rect", 0.0, 1e-8, 1e-3)
    want = sorted(np.ravel_multi_index(k, n) for k in bins)
    np.testing.assert_array_equal(out["located"], want)
    order = np.argsort([np.ravel_multi_index(k, n) for k in bins])
    np.testing.assert_allclose(out["amplitudes"], amps[order], rtol=1e-10)


@pytest.mark.parametrize("p_fa", [1e-3, 1e-6])
def test_threshold_is_the_exponential_quantile(p_fa):
    ws = O.bartlett_window((128, 32), "cheb", 70.0)
    g = O.bartlett_gamma(ws, 2.0, p_fa)
    energy = math.prod(float(np.sum(w ** 2)) for w in ws)
    # P(Exp(mean 2 energy) > g) = p_fa
    assert math.exp(-g / (2.0 * energy)) == pytest.approx(p_fa, rel=1e-12)
