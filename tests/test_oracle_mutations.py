"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin fails.

Each case swaps one oracle function for a subtly wrong version (a transposed
operand, a dropped term, a wrong sign or index) and runs the pin that must
catch it.  This shows the pins are sharp enough to notice such slips.
"""
import importlib
import math

import numpy as np
import pytest

import oracle as O
import oracle.pipeline as orsft
import oracle.windows as owin
import oracle.design as odes
import tests.test_oracle_pins as pins
import tests.test_oracle_refine as rpins
import tests.test_oracle_bartlett as bpins
import tests.test_oracle_estimate as epins


def _perm_inverse(y, sigma_row):
    idx = [(O.inverse_mod(int(s), nd) * np.arange(nd)) % nd for s, nd in zip(sigma_row, y.shape)]
    return y[np.ix_(*idx)]


def _alias_wrong_axis(z, b):
    shape = []
    for nd, bd in zip(z.shape, b):
        shape += [bd, nd // bd]
    return z.reshape(shape).sum(axis=tuple(range(0, 2 * z.ndim, 2)))


def _reverse_with_sigma(plan, l, j):
    return [(int(plan.sigma[l, d]) * (int(j[d]) * plan.m[d] + np.arange(plan.m[d]))) % plan.n[d]
            for d in range(plan.ndim)]


def _flat_conj(n, m, kind, atten_db, support=None):
    return np.conj(_ORIG_FLAT(n, m, kind, atten_db, support))


def _beta_no_square(wbars, ws, sigma_row):
    out = 1.0
    for wbar, w, s in zip(wbars, ws, sigma_row):
        n = len(w)
        out *= float(np.sum(np.abs(wbar) * w[(int(s) * np.arange(n)) % n] ** 2))
    return out


def _median_no_wsum(plan, spectra, located):
    saved = plan.wsum
    plan.wsum = 1.0
    try:
        return _ORIG_EST(plan, spectra, located)
    finally:
        plan.wsum = saved


def _mapping_off_by_one(plan, l, i):
    return tuple(((int(plan.sigma[l, d]) * int(i[d]) + 1) % plan.n[d]) // plan.m[d]
                 for d in range(plan.ndim))


_ORIG_FLAT = owin.flat_window
_ORIG_EST = orsft.estimate_amplitudes
_ORIG_GRAD = O.refine_grad
_ORIG_FIELD = O.tone_field
_ORIG_BARTLETT = O.bartlett
# the package re-exports the function bartlett under the module's own name: reach the module itself
obart = importlib.import_module("oracle.bartlett")


def _grad_no_j(plan, cube, freqs, amps):          # dE/da_im taken along the real direction
    gf, gre, _ = _ORIG_GRAD(plan, cube, freqs, amps)
    return gf, gre, gre


def _grad_freq_sign(plan, cube, freqs, amps):     # exp(-j 2 pi f t) differentiated as exp(+j ...)
    gf, gre, gim = _ORIG_GRAD(plan, cube, freqs, amps)
    return -gf, gre, gim


def _grad_dims_swapped(plan, cube, freqs, amps):  # frequency gradient of the wrong dimension
    gf, gre, gim = _ORIG_GRAD(plan, cube, freqs, amps)
    return gf[:, ::-1], gre, gim


def _field_conj(shape, freqs, amps):              # tones synthesised with the conjugate phase
    return _ORIG_FIELD(shape, -np.asarray(freqs), amps)


def _gamma_no_square(ws, noise_var, p_fa):        # ||w||_1 in place of ||w||_2^2
    energy = 1.0
    for w in ws:
        energy *= float(np.sum(np.abs(w)))
    return -noise_var * energy * math.log(p_fa)


def _dense_gain_squared(*args, **kwargs):         # amplitudes over (sum w)^2 instead of sum w
    out = _ORIG_BARTLETT(*args, **kwargs)
    gain = math.prod(float(np.sum(w)) for w in out["windows"])
    out["amplitudes"] = out["amplitudes"] / gain
    return out

def _floor_upper_median(power, pfa1):          # rank B // 2 in place of floor((B - 1) / 2)
    flat = np.sort(np.asarray(power, dtype=np.float64).reshape(-1))
    return -flat[flat.size // 2] / math.log(2.0) * math.log(pfa1)


def _floor_no_ln2(power, pfa1):                # the median taken as the mean itself
    flat = np.sort(np.asarray(power, dtype=np.float64).reshape(-1))
    return -flat[(flat.size - 1) // 2] * math.log(pfa1)


def _floor_from_mean(power, pfa1):             # sample mean in place of median / ln 2
    return -float(np.mean(power)) * math.log(pfa1)


def _spectrum_at_sigma(plan, r, pairs, rows_per_chunk=0):   # weights indexed with sigma, not sigma^-1
    saved = plan.sigma_inv
    plan.sigma_inv = plan.sigma
    try:
        return _ORIG_SPEC_AT(plan, r, pairs, rows_per_chunk)
    finally:
        plan.sigma_inv = saved


_ORIG_SPEC_AT = orsft.spectrum_at

CASES = [
    ("permute with sigma^-1", [(orsft, "permute", _perm_inverse), (O, "permute", _perm_inverse)],
     lambda: pins.test_permutation_property((16, 8), (3, 7))),
    ("alias over the wrong axis", [(orsft, "alias", _alias_wrong_axis), (O, "alias", _alias_wrong_axis)],
     lambda: pins.test_aliasing_property((16, 32), (4, 8))),
    ("reverse map with sigma", [(orsft, "reverse_map", _reverse_with_sigma), (O, "reverse_map", _reverse_with_sigma)],
     lambda: pins.test_reversibility_and_distinctiveness_exhaustive(16)),
    ("conjugated flat window", [(orsft, "flat_window", _flat_conj), (owin, "flat_window", _flat_conj),
                                (O, "flat_window", _flat_conj)],
     lambda: pins.test_ideal_flat_window_is_boxcar(64, 8)),
    ("beta without the square", [(orsft, "beta_sigma", _beta_no_square), (odes, "beta_sigma", _beta_no_square)],
     pins.test_noise_only_power_is_exponential),
    ("estimate without the pre-window gain", [(orsft, "estimate_amplitudes", _median_no_wsum)],
     lambda: pins.test_exact_recovery_noise_free((64, 32), (8, 8), 6, 4)),
    ("mapping off by one", [(orsft, "mapping", _mapping_off_by_one), (O, "mapping", _mapping_off_by_one)],
     lambda: pins.test_reversibility_and_distinctiveness_exhaustive(16)),
    ("refinement: amplitude gradient without j", [(O, "refine_grad", _grad_no_j)],
     lambda: rpins.test_gradient_matches_central_differences()),
    ("refinement: frequency gradient with the wrong sign", [(O, "refine_grad", _grad_freq_sign)],
     lambda: rpins.test_gradient_matches_central_differences()),
    ("refinement: frequency gradient of the other dimension", [(O, "refine_grad", _grad_dims_swapped)],
     lambda: rpins.test_gradient_matches_central_differences()),
    ("refinement: tones with the conjugate phase", [(O, "tone_field", _field_conj)],
     lambda: rpins.test_tone_field_is_the_sum_of_exponentials()),
    ("dense detector: threshold without the square", [(obart, "bartlett_gamma", _gamma_no_square)],
     lambda: bpins.test_noise_only_power_is_exponential_and_pfa_holds()),
    ("dense detector: amplitude over the squared gain", [(O, "bartlett", _dense_gain_squared)],
     lambda: bpins.test_exact_recovery_of_on_grid_tones()),
    ("noise floor: upper median", [(orsft, "noise_floor_gamma", _floor_upper_median),
                                   (O, "noise_floor_gamma", _floor_upper_median)],
     epins.test_noise_floor_rank_is_the_lower_median),
    ("noise floor: median without ln 2", [(orsft, "noise_floor_gamma", _floor_no_ln2),
                                          (O, "noise_floor_gamma", _floor_no_ln2)],
     lambda: epins.test_noise_floor_threshold_closed_form(256, 0.01)),
    ("noise floor: the mean in place of the median", [(orsft, "noise_floor_gamma", _floor_from_mean),
                                                      (O, "noise_floor_gamma", _floor_from_mean)],
     epins.test_estimate_mode_detects_strong_tones),
    ("sampled spectrum: weights of sigma", [(orsft, "spectrum_at", _spectrum_at_sigma),
                                            (O, "spectrum_at", _spectrum_at_sigma)],
     lambda: epins.test_spectrum_at_equals_fft_of_fold((32, 16), (8, 4))),
]


@pytest.mark.parametrize("name,patches,check", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(monkeypatch, name, patches, check):
    for mod, attr, fn in patches:
        monkeypatch.setattr(mod, attr, fn)
    with pytest.raises(AssertionError):
        check()
