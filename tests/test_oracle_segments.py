"""Pins of the oracle's segment mode (§III-C: each loop processes its own data segment of
the signal model of §IV-A).

* With the same cube in every segment the result is the single-cube RSFT.
* With independent noise-only segments, a location's votes are a sum of L independent
  Bernoulli(P-bar_fa1) draws (its bucket in loop l is detected with probability
  P-bar_fa1 exactly: the power is exponential with mean sigma_n^2 beta(sigma_l) and
  gamma_l = -sigma_n^2 beta(sigma_l) ln P-bar_fa1), so the located fraction is the
  binomial tail P(Bin(L, P-bar_fa1) > mu).
"""
import math

import numpy as np
from scipy.stats import binom

import oracle as O
import rsft_inputs as ri


def test_identical_segments_reduce_to_single_cube_mode():
    n, b, loops = (32, 64), (8, 8), 6
    plan = O.make_plan(n, b, loops, seed=3, pfa1=0.05, mu=2)
    tg = ri.draw_targets(n, 3, "offgrid", 12, (15.0, 20.0), int(np.prod(b)))
    x = ri.tone_cube(n, tg, 1.0, 12).astype(np.complex128)
    one = O.rsft(plan, x)
    seg = O.rsft(plan, [x] * loops)
    np.testing.assert_array_equal(seg["votes"], one["votes"])
    np.testing.assert_array_equal(seg["located"], one["located"])
    np.testing.assert_allclose(seg["amplitudes"], one["amplitudes"], rtol=0, atol=0)


def test_noise_only_segments_give_binomial_vote_tail():
    n, b, loops, nv, pfa1, mu = (64, 64), (8, 8), 8, 2.0, 0.1, 2
    plan = O.make_plan(n, b, loops, seed=41, atten_db=60.0, noise_var=nv, pfa1=pfa1, mu=mu)
    expect = binom.sf(mu, loops, pfa1)
    fracs, zero = [], []
    for frame in range(24):
        segs = [ri.tone_cube(n, None, nv, 90000 + 100 * frame + s).astype(np.complex128) for s in range(loops)]
        out = O.rsft(plan, segs, estimate=False, keep=False)
        fracs.append(len(out["located"]) / float(np.prod(n)))
        zero.append(np.mean(out["votes"] == 0))
    # frames are independent: compare frame means with standard errors from the frames
    for got, want in ((np.asarray(fracs), expect), (np.asarray(zero), binom.pmf(0, loops, pfa1))):
        se = got.std(ddof=1) / math.sqrt(len(got))
        assert abs(got.mean() - want) < 5 * se + 1e-3 * want, (got.mean(), want, se)
