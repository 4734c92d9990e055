"""Seeded synthetic inputs for the RSFT hot path.

This module draws test and benchmark cubes from the signal model of the paper
(§IV-A, eq. (sig_model) and eq. (sinusoid)): a sum of K complex exponentials
with complex amplitudes, plus circular complex white Gaussian noise, extended to
D dimensions by taking one frequency per dimension (§III-C).  It holds none of
the RSFT arithmetic (no windows, permutations, folding, thresholds), so both the
CUDA-path tests and the CPU oracle can read the same cubes from here.

Every draw is keyed by an explicit integer seed, and the noise is generated in
fixed-size chunks, each from its own keyed generator, so a cube is identical on
any machine and with any memory budget.

The workloads of the benchmark configurations live in ``WORKLOADS``.  Tone power
is specified as a per-tone SNR "after the bucket FFT" read with rectangular
coherent gain B: per-sample SNR = SNR_dB - 10 log10(B) (the paper's own SNR is
per sample, §IV-A; the reading is recorded in the design notes).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

__all__ = [
    "Targets", "Workload", "WORKLOADS", "draw_targets", "tone_cube",
    "workload_frame", "frame_seed", "segment_cubes",
    "SrurSystem", "SrurTarget", "TABLE_IV", "srur_frequencies", "srur_bursts", "srur_amplitudes",
]

_CHUNK = 1 << 20  # elements per noise chunk (fixed: part of the cube definition)


@dataclasses.dataclass
class Targets:
    """Tone parameters: ``freqs`` K x D in cycles/sample, ``amps`` K complex."""
    freqs: np.ndarray
    amps: np.ndarray
    snr_db: np.ndarray

    def grid_index(self, shape: Sequence[int]) -> np.ndarray:
        n = np.asarray(shape, dtype=np.int64)
        return np.rint(self.freqs * n).astype(np.int64) % n


@dataclasses.dataclass(frozen=True)
class Workload:
    """One benchmark configuration (shapes and signal recipe only)."""
    name: str
    shape: tuple
    buckets: tuple
    loops: int
    atten_db: float
    p_fa: float
    k_range: tuple          # (k_min, k_max) inclusive
    snr_db: tuple           # (lo, hi) per-tone SNR after the bucket FFT
    kind: str               # "ongrid" | "offgrid"
    amp_model: str          # "unit" | "rayleigh" | "loguniform"
    min_sep_bins: float = 0.0
    flat_support: tuple | None = None
    noise_var: float = 1.0
    index: int = 0
    design_k: int = 0       # sparsity budget of the threshold design (0: k_range[1])

    @property
    def k_design(self) -> int:
        return self.design_k or self.k_range[1]


WORKLOADS = {
    "c1_2d_256": Workload("c1_2d_256", (256, 256), (16, 16), 8, 60.0, 1e-4,
                          (8, 8), (10.0, 10.0), "ongrid", "unit",
                          flat_support=(64, 64), index=0),
    "c2_3d_radar": Workload("c2_3d_radar", (1024, 256, 64), (64, 32, 8), 12,
                            80.0, 1e-6, (32, 32), (5.0, 25.0), "offgrid",
                            "rayleigh", index=1),
    # B = 128 buckets: K eta_m >= B for K = 64 (Remark 2), so the design budget is K = 8
    "c3_small": Workload("c3_small", (256, 128, 16), (16, 8, 1), 10, 60.0,
                         1e-5, (4, 64), (5.0, 25.0), "offgrid", "rayleigh",
                         index=2, design_k=8),
    "c3_mid": Workload("c3_mid", (512, 256, 32), (32, 16, 2), 10, 60.0, 1e-5,
                       (4, 64), (5.0, 25.0), "offgrid", "rayleigh", index=2),
    "c3_large": Workload("c3_large", (1024, 256, 64), (64, 16, 4), 10, 60.0,
                         1e-5, (4, 64), (5.0, 25.0), "offgrid", "rayleigh",
                         index=2),
    "c4_2d_4096": Workload("c4_2d_4096", (4096, 4096), (128, 128), 16, 60.0,
                           1e-6, (100, 100), (0.0, 30.0), "offgrid",
                           "loguniform", min_sep_bins=4.0, index=3),
    "c5_4d": Workload("c5_4d", (512, 512, 64, 32), (32, 32, 8, 4), 16, 80.0,
                      1e-7, (256, 256), (0.0, 20.0), "offgrid", "rayleigh",
                      index=4),
}


def frame_seed(workload: Workload, frame: int) -> int:
    """Seed of one frame of a workload: configuration index x 1000 + frame."""
    return int(workload.index) * 1000 + int(frame)


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


def draw_targets(shape: Sequence[int], k: int, kind: str, seed: int,
                 snr_db: tuple, buckets_total: int, noise_var: float = 1.0,
                 amp_model: str = "rayleigh", min_sep_bins: float = 0.0) -> Targets:
    """Draw K tones.

    kind "ongrid": distinct integer frequencies f = k/N_d; "offgrid": continuous
    uniform in [0, 1) per dimension, optionally rejection-sampled to a circular
    L-infinity separation of at least ``min_sep_bins`` bins.  Amplitudes:
    "unit" |a| = 1 (noise_var then carries the SNR), "rayleigh" a ~ CN(0, s2)
    (Swerling-I, §IV-A and §VI-A), "loguniform" |a|^2 = s2 with uniform phase;
    s2 = noise_var * 10^(SNR/10) / B with SNR uniform in ``snr_db`` (dB).
    """
    rng = _rng(seed, 1)
    n = np.asarray(shape, dtype=np.int64)
    d = len(shape)
    freqs = np.zeros((k, d))
    if kind == "ongrid":
        seen = set()
        i = 0
        while i < k:
            g = tuple(int(rng.integers(0, nd)) for nd in n)
            if g in seen:
                continue
            seen.add(g)
            freqs[i] = np.asarray(g) / n
            i += 1
    elif kind == "offgrid":
        i = 0
        tries = 0
        while i < k:
            f = rng.random(d)
            tries += 1
            if tries > 100000 * max(k, 1):
                raise RuntimeError("cannot place tones with the requested separation")
            if min_sep_bins > 0 and i > 0:
                diff = np.abs(freqs[:i] - f) * n
                diff = np.minimum(diff, n - diff)
                if np.any(np.max(diff, axis=1) < min_sep_bins):
                    continue
            freqs[i] = f
            i += 1
    else:
        raise ValueError(kind)
    snr = rng.uniform(snr_db[0], snr_db[1], size=k)
    s2 = noise_var * 10.0 ** (snr / 10.0) / float(buckets_total)
    phase = np.exp(2j * np.pi * rng.random(k))
    if amp_model == "unit":
        amps = phase.astype(np.complex128)
    elif amp_model == "rayleigh":
        g = (rng.standard_normal(k) + 1j * rng.standard_normal(k)) / math.sqrt(2.0)
        amps = np.sqrt(s2) * g
    elif amp_model == "loguniform":
        amps = np.sqrt(s2) * phase
    else:
        raise ValueError(amp_model)
    return Targets(freqs=freqs, amps=amps, snr_db=snr)


def tone_cube(shape: Sequence[int], targets: Targets | None, noise_var: float,
              seed: int, out: np.ndarray | None = None) -> np.ndarray:
    """Return a complex64 cube x[s] = sum_k a_k exp(j 2 pi sum_d f_kd s_d) + n[s].

    n ~ CN(0, noise_var I).  Tones are evaluated in float64 as an outer product
    over a split of the dimensions (a matrix product per chunk of leading rows)
    and rounded once to complex64.
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    total = int(np.prod(shape))
    if out is None:
        out = np.empty(shape, dtype=np.complex64)
    flat = out.reshape(-1)
    split = max(1, d // 2) if d > 1 else 1
    left = int(np.prod(shape[:split])) if d > 1 else 1
    right = total // left
    have_tones = targets is not None and len(targets.amps) > 0
    if have_tones:
        kk = len(targets.amps)
        right_fac = np.ones((kk, 1), dtype=np.complex128)
        for dd in range(split if d > 1 else 0, d):
            s = np.arange(shape[dd])
            e = np.exp(2j * np.pi * np.outer(targets.freqs[:, dd], s))
            right_fac = (right_fac.reshape(kk, -1, 1) * e.reshape(kk, 1, -1)).reshape(kk, -1)
    rows_per_chunk = max(1, _CHUNK // right)
    sd = math.sqrt(noise_var / 2.0)
    for c0 in range(0, left, rows_per_chunk):
        c1 = min(left, c0 + rows_per_chunk)
        rows = np.arange(c0, c1)
        block = np.zeros((c1 - c0, right), dtype=np.complex128)
        if have_tones:
            left_fac = np.tile(targets.amps.astype(np.complex128), (c1 - c0, 1))
            if d > 1:
                idx = np.unravel_index(rows, shape[:split])
                for dd in range(split):
                    left_fac = left_fac * np.exp(2j * np.pi * np.outer(idx[dd], targets.freqs[:, dd]))
            block += left_fac @ right_fac
        if noise_var > 0:
            rng = _rng(seed, 2, c0)
            nz = rng.standard_normal((c1 - c0, right, 2))
            block += sd * (nz[..., 0] + 1j * nz[..., 1])
        flat[c0 * right:c1 * right] = block.reshape(-1)
    return out


def workload_frame(name: str, frame: int = 0, shape: Sequence[int] | None = None,
                   with_noise: bool = True):
    """Return (cube complex64, Targets, Workload) for one frame of a workload."""
    wl = WORKLOADS[name]
    seed = frame_seed(wl, frame)
    shp = tuple(shape) if shape is not None else wl.shape
    btot = int(np.prod(wl.buckets))
    rng = _rng(seed, 0)
    k = int(rng.integers(wl.k_range[0], wl.k_range[1] + 1))
    noise_var = wl.noise_var
    if wl.amp_model == "unit":
        # unit-amplitude tones: the SNR sets the noise level instead
        noise_var = float(btot) / 10.0 ** (wl.snr_db[0] / 10.0)
    tg = draw_targets(shp, k, wl.kind, seed, wl.snr_db, btot, noise_var=noise_var,
                      amp_model=wl.amp_model, min_sep_bins=wl.min_sep_bins)
    cube = tone_cube(shp, tg, noise_var if with_noise else 0.0, seed)
    return cube, tg, wl, noise_var


def segment_cubes(shape: Sequence[int], targets: Targets, noise_var: float, seed: int, segments: int,
                  buckets_total: int) -> list:
    """One cube per data segment (the signal model of §IV-A): the tones keep their
    frequencies, their complex amplitudes are redrawn for every segment as
    b_{i,s} ~ CN(0, sigma_bi^2) (Swerling-I), with sigma_bi^2 set from the target's SNR
    (read after the B-point bucket FFT, like ``draw_targets``), and every segment gets its
    own noise.  Seeds: (seed, segment) keyed."""
    out = []
    sb2 = noise_var * 10.0 ** ((np.asarray(targets.snr_db, dtype=np.float64) - 10.0 * np.log10(buckets_total)) / 10.0)
    for s in range(segments):
        rng = np.random.default_rng([seed, 7919, s])
        amps = (rng.standard_normal(len(sb2)) + 1j * rng.standard_normal(len(sb2))) * np.sqrt(sb2 / 2.0)
        tg = Targets(targets.freqs, amps, targets.snr_db)
        out.append(tone_cube(shape, tg, noise_var, seed * 1000 + 17 * s + 1))
    return out


# ---------------------------------------------------------------- SRUR radar cubes (§VI)

@dataclasses.dataclass(frozen=True)
class SrurSystem:
    """The short-range ubiquitous radar of §VI-B (Table III): an LFMCW waveform de-chirped
    in analogue and IQ-sampled on every element of a half-wavelength uniform linear array."""
    range_bins: int = 2048      # R: fast-time samples per repetition interval
    elements: int = 64          # N: receiving elements
    ris: int = 32               # M: repetition intervals per burst
    wavelength: float = 0.03    # lambda (m)
    c: float = 3.0e8            # propagation speed (m/s)
    bandwidth: float = 150.0e6  # B_w (Hz)
    t_p: float = 5.0e-5         # T_p: repetition interval (s)
    r_max: float = 1.5e3        # maximum range (m)
    chirp_rate: float = 3.0e12  # rho (Hz/s)
    f_s: float = 41.0e6         # IQ sampling frequency (Hz)

    @property
    def shape(self) -> tuple:
        """Cube layout (range sample, element, repetition interval): the R x N x M data cube."""
        return (self.range_bins, self.elements, self.ris)


@dataclasses.dataclass(frozen=True)
class SrurTarget:
    """One point target: range (m), closing velocity (m/s), direction of arrival from the
    array normal (degrees) and per-sample SNR (dB, the paper's SNR_i of §IV-A)."""
    range_m: float
    velocity: float
    doa_deg: float
    snr_db: float


# Table IV: four targets; targets 3 and 4 differ only by 4 degrees of DOA.  "equal": every
# target at -10 dB; "mixed": 0, -10, -20, -20 dB.
TABLE_IV = {
    "equal": (SrurTarget(1000.0, 100.0, 30.0, -10.0), SrurTarget(500.0, 50.0, 0.0, -10.0),
              SrurTarget(350.0, 240.0, -16.0, -10.0), SrurTarget(350.0, 240.0, -20.0, -10.0)),
    "mixed": (SrurTarget(1000.0, 100.0, 30.0, 0.0), SrurTarget(500.0, 50.0, 0.0, -10.0),
              SrurTarget(350.0, 240.0, -16.0, -20.0), SrurTarget(350.0, 240.0, -20.0, -20.0)),
}


def srur_frequencies(system: SrurSystem, targets: Sequence[SrurTarget]) -> np.ndarray:
    """K x 3 frequencies in cycles per sample along (range sample, element, RI), in [0, 1).

    Eq. (s_u): the de-chirp leaves the beat frequency f_r = 2 rho r / c in fast time (sampled
    at f_s) and the Doppler frequency f_d = 2 v / lambda, whose phase advances by f_d T_p per
    repetition interval; half-wavelength element spacing advances the phase by pi sin(theta)
    per element, sin(theta) / 2 cycles."""
    f = np.zeros((len(targets), 3))
    for k, t in enumerate(targets):
        f_r = 2.0 * system.chirp_rate * t.range_m / system.c
        f_d = 2.0 * t.velocity / system.wavelength
        f[k] = (f_r / system.f_s, 0.5 * math.sin(math.radians(t.doa_deg)), f_d * system.t_p)
    return f - np.floor(f)


def srur_bursts(system: SrurSystem, targets: Sequence[SrurTarget], bursts: int, seed: int,
                amplitudes: np.ndarray | None = None, noise_var: float = 1.0):
    """T bursts of the de-chirped array signal of eq. (r_i), as complex64 IQ cubes of
    ``system.shape``:

        r[tau, i, v] = sum_k a_k(s) exp(j 2 pi (f_r tau / f_s + i sin(theta_k) / 2 + f_d v T_p)) + n,

    n ~ CN(0, noise_var).  Swerling-I amplitudes (§VI-A): a_k(s) ~ CN(0, noise_var 10^(SNR_k/10)),
    static within burst s and independent between bursts, unless ``amplitudes`` ([T][K]) fixes
    them.  Returns (cubes, freqs [K][3], amplitudes [T][K]); each burst is one data segment of
    the segment mode (one loop per burst).  Seeds: (seed, burst) keyed."""
    freqs = srur_frequencies(system, targets)
    snr = np.asarray([t.snr_db for t in targets], dtype=np.float64)
    # a noise-free cube (noise_var = 0) keeps the amplitudes of unit noise
    amps = (srur_amplitudes(targets, bursts, seed, noise_var if noise_var > 0 else 1.0) if amplitudes is None
            else np.asarray(amplitudes, dtype=np.complex128))
    cubes = [tone_cube(system.shape, Targets(freqs, amps[s], snr), noise_var, seed * 1000 + 31 * s + 3)
             for s in range(bursts)]
    return cubes, freqs, amps


def srur_amplitudes(targets: Sequence[SrurTarget], bursts: int, seed: int, noise_var: float = 1.0) -> np.ndarray:
    """[T][K] Swerling-I amplitudes: a_k(s) ~ CN(0, noise_var 10^(SNR_k / 10)), one draw per
    burst (keyed by (seed, burst))."""
    s2 = noise_var * 10.0 ** (np.asarray([t.snr_db for t in targets], dtype=np.float64) / 10.0)
    out = np.empty((bursts, len(s2)), dtype=np.complex128)
    for s in range(bursts):
        rng = _rng(seed, 11, s)
        out[s] = (rng.standard_normal(len(s2)) + 1j * rng.standard_normal(len(s2))) * np.sqrt(s2 / 2.0)
    return out
