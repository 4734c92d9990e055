"""Pins of the oracle's bucket-domain refinement loss and gradient.

The analytic gradient (chain rule through the linear fold) is checked against central
finite differences of the loss in FP64, parameter by parameter; the loss is zero at the
true tones of a noise-free cube; and the tone field is checked against a dense sum of
complex exponentials written out directly.
"""
import numpy as np
import pytest

import oracle as O


def _case():
    n, b, loops = (32, 16), (8, 4), 3
    plan = O.make_plan(n, b, loops, seed=19, atten_db=50.0, pfa1=0.05, mu=1)
    true_f = np.array([[0.2031, 0.4106], [0.6719, 0.0833]])
    true_a = np.array([1.3 - 0.4j, 0.6 + 0.9j])
    cube = O.tone_field(n, true_f, true_a)
    rng = np.random.default_rng(4)
    cube = cube + 0.05 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    f0 = true_f + np.array([[0.004, -0.003], [-0.002, 0.005]])
    a0 = true_a * (0.9 + 0.1j)
    return plan, cube, f0, a0, true_f, true_a


def test_tone_field_is_the_sum_of_exponentials():
    f = np.array([[0.1, 0.7]])
    a = np.array([2.0 - 1.0j])
    got = O.tone_field((4, 8), f, a)
    for t0 in range(4):
        for t1 in range(8):
            assert abs(got[t0, t1] - a[0] * np.exp(2j * np.pi * (0.1 * t0 + 0.7 * t1))) < 1e-12


def test_loss_vanishes_at_the_true_noise_free_tones():
    plan, _, _, _, tf, ta = _case()
    cube = O.tone_field(plan.n, tf, ta)
    assert O.refine_loss(plan, cube, tf, ta) < 1e-18 * O.refine_loss(plan, cube, tf * 0.0, ta)


def test_gradient_matches_central_differences():
    plan, cube, f0, a0, _, _ = _case()
    gf, gre, gim = O.refine_grad(plan, cube, f0, a0)
    h = 1e-6
    for k in range(len(a0)):
        for d in range(2):
            fp, fm = f0.copy(), f0.copy()
            fp[k, d] += h
            fm[k, d] -= h
            fd = (O.refine_loss(plan, cube, fp, a0) - O.refine_loss(plan, cube, fm, a0)) / (2 * h)
            assert fd == pytest.approx(gf[k, d], rel=1e-6, abs=1e-6 * np.abs(gf).max())
        for unit, g in ((1.0, gre[k]), (1j, gim[k])):
            ap, am = a0.copy(), a0.copy()
            ap[k] += h * unit
            am[k] -= h * unit
            fd = (O.refine_loss(plan, cube, f0, ap) - O.refine_loss(plan, cube, f0, am)) / (2 * h)
            assert fd == pytest.approx(g, rel=1e-6, abs=1e-6 * max(abs(gre).max(), abs(gim).max()))
