"""Windows (oracle side).

Pre-permutation window: the Dolph-Chebyshev window named in §III-C.1 (citing
Harris 1978), symmetric (Claim 1's proof relies on symmetry) and scaled to a
peak of 1.  Its DTFT is e^{-j w (n-1)/2} T_{n-1}(x0 cos(w/2)) with
x0 = cosh(acosh(10^{A/20}) / (n-1)); sampling that at w = 2 pi k / n and taking
the inverse DFT gives the n taps.

Flat window: §IV-B fixes only its pass band (width 2 pi / B) and its length (N);
§V says it is built from the same Chebyshev window with pass band 1/B.  The
reading used here: the pass band of bucket k is the M = N/B permuted bins
[kM, (k+1)M) (the floor mapping of Def. 3 and Def. 4), realised in time as the
Dirichlet sum  sum_{p<M} e^{-j 2 pi p t / N}, tapered by an odd-length
Chebyshev window centred circularly at t = 0 (support S - 1 taps), and scaled
so the response in the middle of the pass band is exactly 1.  "ideal" drops the
taper (an exact frequency boxcar).
"""
from __future__ import annotations

import numpy as np


def chebyshev_poly(order: int, x: np.ndarray) -> np.ndarray:
    """Chebyshev polynomial of the first kind T_order(x) for real x."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(order * np.arccos(x[inside]))
    hi = x > 1.0
    out[hi] = np.cosh(order * np.arccosh(x[hi]))
    lo = x < -1.0
    sign = -1.0 if order % 2 else 1.0
    out[lo] = sign * np.cosh(order * np.arccosh(-x[lo]))
    return out


def chebyshev_window(n: int, atten_db: float) -> np.ndarray:
    """Dolph-Chebyshev window of length n with side lobes at -atten_db dB."""
    if n < 1:
        raise ValueError("window length must be >= 1")
    if n == 1:
        return np.ones(1)
    order = n - 1
    x0 = np.cosh(np.arccosh(10.0 ** (atten_db / 20.0)) / order)
    k = np.arange(n)
    amp = chebyshev_poly(order, x0 * np.cos(np.pi * k / n))
    spectrum = amp * np.exp(-1j * np.pi * k * (n - 1) / n)
    w = np.real(np.fft.ifft(spectrum))
    return w / np.max(w)


def pre_window(n: int, kind: str, atten_db: float) -> np.ndarray:
    """Pre-permutation window w_d of one dimension (§III-A, §III-C.1)."""
    if kind == "rect":
        return np.ones(n)
    if kind == "cheb":
        return chebyshev_window(n, atten_db)
    raise ValueError(kind)


def flat_window(n: int, m: int, kind: str, atten_db: float, support: int | None = None) -> np.ndarray:
    """Flat window w-bar_d of one dimension: pass band = m permuted bins [0, m).

    w-bar(t) = g * c(t) * sum_{p=0}^{m-1} exp(-j 2 pi p t / n),  t in [n].
    kind "ideal": c = 1.  kind "cheb": c = Chebyshev window of odd length
    S - 1 (S = ``support``, default n) centred at t = 0 modulo n.
    g makes the response at pass-band offset floor(m/2) equal to 1.
    """
    t = np.arange(n)
    dirichlet = np.zeros(n, dtype=np.complex128)
    for p in range(m):
        dirichlet += np.exp(-2j * np.pi * p * t / n)
    if kind == "ideal":
        taper = np.ones(n)
    elif kind == "cheb":
        s = n if support is None else int(support)
        if s < 2 or s > n or s % 2:
            raise ValueError("flat support must be even and in [2, n]")
        half = (s - 2) // 2
        c = chebyshev_window(2 * half + 1, atten_db)
        taper = np.zeros(n)
        taper[np.arange(-half, half + 1) % n] = c
    else:
        raise ValueError(kind)
    raw = taper * dirichlet
    response = np.fft.fft(raw) / n
    g = 1.0 / np.real(response[(-(m // 2)) % n])
    return g * raw


def flat_gain(wbar: np.ndarray) -> np.ndarray:
    """G(u) = DFT(w-bar)[u] / N: gain of bucket k for permuted bin q at u = kM - q."""
    return np.fft.fft(wbar) / len(wbar)


def dtft_magnitude(w: np.ndarray, nu: float) -> float:
    """|sum_t w(t) e^{-j 2 pi nu t / n}| at a fractional bin nu (direct sum)."""
    n = len(w)
    return float(np.abs(np.sum(w * np.exp(-2j * np.pi * nu * np.arange(n) / n))))


def window_6db_bins(w: np.ndarray) -> float:
    """6.0-dB bandwidth of a window in DFT bins (Harris 1978; eta_m of Claim 3).

    Full width of the main lobe where the amplitude response is half its peak:
    step out from nu = 0 in 1/16-bin steps until the response drops below one
    half, then bisect the crossing on the direct DTFT.
    """
    peak = dtft_magnitude(w, 0.0)
    lo, hi = 0.0, None
    nu = 0.0
    while nu < len(w):
        nu += 1.0 / 16.0
        if dtft_magnitude(w, nu) < 0.5 * peak:
            hi = nu
            break
        lo = nu
    if hi is None:
        return float(len(w))
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if dtft_magnitude(w, mid) < 0.5 * peak:
            hi = mid
        else:
            lo = mid
    return 2.0 * 0.5 * (lo + hi)
