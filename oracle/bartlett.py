"""Dense Bartlett detector of Appendix A (Algorithm 2) with one data segment.

The comparison system of the RSFT: window the whole N-D cube, take its full N-point
N-D DFT, and run a Neyman-Pearson test on every bin's power.  With one segment
(T = 1) the test statistic is the bin power |u-hat_k|^2 itself, which under H0 is
exponential with mean sigma_n^2 beta' (beta' = ||w||^2, the H0 variance stated in
Appendix A), so the exact NP threshold for a per-bin false-alarm probability P_fa is
gamma = -sigma_n^2 ||w||^2 ln P_fa.  Detections are reported in ascending row-major
order; the amplitude of a detected bin is u-hat_k / prod_d sum_t w_d(t), the complex
amplitude of an on-grid tone at that bin.

Test infrastructure only (see the package docstring); FP64 throughout.
"""
from __future__ import annotations

import math

import numpy as np

from .windows import pre_window


def bartlett_window(n, window: str = "cheb", atten_db: float = 60.0) -> list[np.ndarray]:
    """Per-dimension windows w_d (the N-D window is their outer product, §III-C)."""
    return [pre_window(int(nd), window, atten_db) for nd in n]


def bartlett_gamma(ws, noise_var: float, p_fa: float) -> float:
    """Exact NP threshold of one segment: -sigma_n^2 ||w||^2 ln P_fa."""
    energy = 1.0
    for w in ws:
        energy *= float(np.sum(np.abs(w) ** 2))
    return -noise_var * energy * math.log(p_fa)


def bartlett(x: np.ndarray, window: str = "cheb", atten_db: float = 60.0, noise_var: float = 1.0,
             p_fa: float = 1e-6) -> dict:
    """Algorithm 2 with T = 1: windowing, N-D FFT, power, NP detection, amplitudes."""
    x = np.asarray(x, dtype=np.complex128)
    ws = bartlett_window(x.shape, window, atten_db)
    w = ws[0]
    for wd in ws[1:]:
        w = np.multiply.outer(w, wd)
    spectrum = np.fft.fftn(w * x)
    power = np.abs(spectrum) ** 2
    gamma = bartlett_gamma(ws, noise_var, p_fa)
    located = np.flatnonzero(power.reshape(-1) > gamma)
    gain = 1.0
    for wd in ws:
        gain *= float(np.sum(wd))
    amplitudes = spectrum.reshape(-1)[located] / gain
    return {"spectrum": spectrum, "power": power, "gamma": gamma, "located": located,
            "amplitudes": amplitudes, "windows": ws}


def bartlett_pd_swerling1(p_fa: float, snr_gain: float) -> float:
    """Detection probability of one segment for a Swerling-I tone on the bin under test.

    With a ~ CN(0, sigma_b^2) the bin is CN(0, sigma_b^2 alpha' + sigma_n^2 beta'), so
    P_d = exp(-gamma / (sigma_b^2 alpha' + sigma_n^2 beta')) = P_fa^(1 / (1 + snr_gain)),
    snr_gain = sigma_b^2 alpha' / (sigma_n^2 beta').
    """
    return p_fa ** (1.0 / (1.0 + snr_gain))
