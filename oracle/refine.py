"""Bucket-domain refinement of off-grid tones (beyond the paper; test infrastructure only).

The RSFT locates frequencies on the N-point grid and estimates their amplitudes (§III).  A
K-tone model theta = {(f_k, a_k)}, f_k in [0, 1)^D cycles per sample, a_k complex, can be
refined against the same data by comparing folded buckets: for every loop l the model cube
s_theta(t) = sum_k a_k exp(j 2 pi sum_d f_kd t_d) goes through the loop's pre-window,
permutation, flat window and aliasing (Algorithm 1, the oracle's ``fold_loop``), and the
loss is the squared bucket residual

    E(theta) = sum_l || F_l - fold_l(s_theta) ||^2,     F_l = fold_l(r).

fold_l is linear, so dE/dtheta = -2 Re sum_l < F_l - fold_l(s_theta), fold_l(ds_theta/dtheta) >
with ds/da_re = e_k, ds/da_im = j e_k, ds/df_kd = a_k (j 2 pi t_d) e_k, e_k(t) = exp(j 2 pi f_k . t).
Everything here is the plain N-point route (synthesise, fold with the oracle's fold, take
inner products) in FP64: slow, for small cubes.
"""
from __future__ import annotations

import numpy as np

from .pipeline import OraclePlan, fold_loop


def tone_field(shape, freqs, amps) -> np.ndarray:
    """s(t) = sum_k a_k exp(j 2 pi f_k . t) on the N-point grid (FP64)."""
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    out = np.zeros(shape, dtype=np.complex128)
    for f, a in zip(np.asarray(freqs, dtype=np.float64), np.asarray(amps, dtype=np.complex128)):
        phase = sum(float(f[d]) * grids[d] for d in range(len(shape)))
        out += a * np.exp(2j * np.pi * phase)
    return out


def refine_loss(plan: OraclePlan, cube: np.ndarray, freqs, amps) -> float:
    """E(theta) = sum_l ||fold_l(r) - fold_l(s_theta)||^2."""
    model = tone_field(plan.n, freqs, amps)
    resid = np.asarray(cube, dtype=np.complex128) - model
    return float(sum(np.sum(np.abs(fold_loop(plan, resid, l)) ** 2) for l in range(plan.loops)))


def refine_grad(plan: OraclePlan, cube: np.ndarray, freqs, amps):
    """(dE/df [K, D], dE/da_re [K], dE/da_im [K]) by the chain rule through the linear fold."""
    freqs = np.asarray(freqs, dtype=np.float64)
    amps = np.asarray(amps, dtype=np.complex128)
    shape = plan.n
    resid = np.asarray(cube, dtype=np.complex128) - tone_field(shape, freqs, amps)
    rl = [fold_loop(plan, resid, l) for l in range(plan.loops)]
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")

    def contract(field):  # -2 Re sum_l < R_l, fold_l(field) >
        return -2.0 * sum(np.real(np.vdot(rl[l], fold_loop(plan, field, l))) for l in range(plan.loops))

    gf = np.zeros(freqs.shape)
    gre = np.zeros(len(amps))
    gim = np.zeros(len(amps))
    for k in range(len(amps)):
        e = np.exp(2j * np.pi * sum(freqs[k, d] * grids[d] for d in range(len(shape))))
        gre[k] = contract(e)
        gim[k] = contract(1j * e)
        for d in range(len(shape)):
            gf[k, d] = contract(amps[k] * 2j * np.pi * grids[d] * e)
    return gf, gre, gim
