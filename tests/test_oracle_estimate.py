"""Pins of the oracle's estimate mode of the first stage, of its sampled bucket spectrum and of
the binomial second-stage design (no GPU).

Estimate mode (§IV-B, eq. (exp), eq. (tpd)): each loop's threshold is the lower median of its
B bucket powers divided by ln 2, times -ln Pfa1.  For B independent exponential powers the
expected number of detections has a closed form, whatever the noise level: with
X_(1) <= ... <= X_(B) the order statistics, k = floor((B - 1) / 2) + 1 and c = -ln Pfa1 / ln 2,
the Renyi representation X_(k) = theta sum_{i <= k} E_i / (B - i + 1) (E_i independent unit
exponentials) and the memorylessness of the B - k larger powers give
    E[#{i : X_i > c X_(k)}] = (B - k) prod_{i=1}^{k} (B - i + 1) / (B - i + c)     (c > 1).
The oracle's threshold function is checked against it on simulated powers, and the whole
oracle on noise-only cubes.

Binomial design (§IV-C, Claims 2-3 read with the exact vote law): on noise-only cubes each
cell's vote count is Binomial(L, Pfa1) because the loops draw sigma independently (Def. 1);
the empirical distribution of the oracle's votes is checked against it, and the Normal form of
Claim 3 is shown to miss the tail that the design targets.
"""
import math

import numpy as np
import pytest
from scipy.stats import beta as beta_dist

import oracle as O
import rsft_inputs as ri


def expected_detections(b: int, pfa1: float) -> float:
    """Closed form above: expected detections among B exponential powers in estimate mode."""
    k = (b - 1) // 2 + 1
    c = -math.log(pfa1) / math.log(2.0)
    log_prod = sum(math.log(b - i + 1) - math.log(b - i + c) for i in range(1, k + 1))
    return (b - k) * math.exp(log_prod)


@pytest.mark.parametrize("b,pfa1", [(256, 0.01), (1024, 1e-3), (255, 0.05)])
def test_noise_floor_threshold_closed_form(b, pfa1):
    rng = np.random.default_rng(b)
    trials = 4000
    counts = np.empty(trials)
    for t in range(trials):
        theta = float(rng.uniform(0.1, 10.0))            # any noise level: the rate does not depend on it
        p = theta * rng.exponential(size=b)
        counts[t] = np.sum(p > O.noise_floor_gamma(p, pfa1))
    expect = expected_detections(b, pfa1)
    se = counts.std(ddof=1) / math.sqrt(trials)
    assert abs(counts.mean() - expect) < 4.5 * se + 1e-12, (counts.mean(), expect, se)
    # the estimate is consistent: at large B the rate approaches Pfa1 itself
    assert abs(expected_detections(1 << 16, pfa1) / (1 << 16) / pfa1 - 1) < 0.02


def test_noise_floor_rank_is_the_lower_median():
    # ranks 0..B-1 ascending; B even takes rank B/2 - 1, B odd the middle one
    for b in (2, 3, 8, 9, 1024):
        p = np.random.default_rng(b).permutation(np.arange(1, b + 1, dtype=np.float64))
        lower = (b - 1) // 2 + 1                          # value of rank floor((B - 1) / 2) is that + 0
        assert O.noise_floor_gamma(p, math.exp(-1.0)) == pytest.approx(lower / math.log(2.0), rel=1e-15)


def test_estimate_mode_on_noise_only_cubes():
    # the whole oracle: rate within the closed form's reach, thresholds near sigma_n^2 beta ln(1/Pfa1),
    # and detections that do not depend on the noise level (scale invariance of the estimate)
    n, b, loops, pfa1 = (64, 128), (16, 16), 16, 0.02
    bt = int(np.prod(b))
    known = O.make_plan(n, b, loops, seed=31, atten_db=60.0, noise_var=2.0, pfa1=pfa1, mu=3)
    est = O.make_plan(n, b, loops, seed=31, atten_db=60.0, noise_var=0.0, pfa1=pfa1, mu=3)
    assert est.estimate_noise and np.all(np.isnan(est.gamma))
    hits, total = 0, 0
    for frame in range(6):
        x = ri.tone_cube(n, None, 2.0, 7000 + frame).astype(np.complex128)
        out = O.rsft(est, x, estimate=False, keep=False)
        ratio = out["gamma"] / known.gamma
        assert np.all(np.abs(ratio - 1) < 6 / (math.log(2) * math.sqrt(bt)))   # median's spread ~ 1/(ln2 sqrt B)
        hits += int(out["detected"].sum())
        total += out["detected"].size
        if frame == 0:
            out10 = O.rsft(est, 10.0 * x, estimate=False, keep=False)
            np.testing.assert_array_equal(out10["detected"], out["detected"])
            np.testing.assert_allclose(out10["gamma"], 100.0 * out["gamma"], rtol=1e-12)
    rate = expected_detections(bt, pfa1) / bt
    lo = beta_dist.ppf(0.0005, hits, total - hits + 1)
    hi = beta_dist.ppf(0.9995, hits + 1, total - hits)
    # buckets of one loop are mildly correlated (overlapping flat-window responses), which widens
    # the spread of the median beyond the independent case: allow a quarter either side
    assert 0.75 * lo <= rate <= 1.25 * hi, (lo, rate, hi)


def test_estimate_mode_detects_strong_tones():
    n, b, loops = (128, 128), (16, 16), 8
    tg = ri.draw_targets(n, 4, "ongrid", 12, (25.0, 25.0), int(np.prod(b)))
    x = ri.tone_cube(n, tg, 1.0, 12).astype(np.complex128)
    est = O.make_plan(n, b, loops, seed=12, noise_var=-1.0, pfa1=1e-3, mu=5)
    out = O.rsft(est, x, estimate=False)
    truth = np.ravel_multi_index(tg.grid_index(n).T, n)
    assert set(truth.tolist()) <= set(out["located"].tolist())
    # the median is robust: four strong tones move the noise floor by a few ranks of 256 (their
    # main lobes and transition bands: ratios 1.0-1.6 here), while a mean would follow their power
    # (ratios 3.2-3.8)
    known = O.make_plan(n, b, loops, seed=12, noise_var=1.0, pfa1=1e-3, mu=5)
    assert np.all(np.abs(out["gamma"] / known.gamma - 1) < 1.0), out["gamma"] / known.gamma


# ----------------------------------------------------------------------------- sampled spectrum

@pytest.mark.parametrize("n,b", [((64,), (8,)), ((32, 16), (8, 4)), ((16, 8, 8), (4, 2, 2)),
                                 ((8, 8, 4, 4), (2, 4, 2, 1))])
def test_spectrum_at_equals_fft_of_fold(n, b):
    loops = 3
    plan = O.make_plan(n, b, loops, seed=5, atten_db=60.0, pfa1=0.1, mu=1)
    rng = np.random.default_rng(3)
    r = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    full = np.stack([np.fft.fftn(O.fold_loop(plan, r, l)) for l in range(loops)])
    pairs = [(l, idx) for l in range(loops) for idx in np.ndindex(*b)]
    got = O.spectrum_at(plan, r, pairs, rows_per_chunk=max(1, n[0] // 4))
    ref = np.array([full[(l,) + tuple(idx)] for l, idx in pairs])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


# ----------------------------------------------------------------------------- binomial design

def test_noise_only_votes_are_binomial():
    # sigma_l independent per loop: a cell's count is Binomial(L, Pfa1) on noise alone.  Every loop
    # folds the same cube, so a frequency's own noise power enters its bucket in every loop; with
    # M = N / B aliases per bucket its share is about 1 / M, and at M = 256 the law holds to a few
    # percent (at M = 16 the tail at mu = 3 is twice the binomial one)
    n, b, loops, pfa1 = (256, 256), (16, 16), 12, 0.05
    counts = []
    for seed in range(4):
        plan = O.make_plan(n, b, loops, seed=100 + seed, atten_db=60.0, noise_var=1.0, pfa1=pfa1, mu=0)
        x = ri.tone_cube(n, None, 1.0, 900 + seed).astype(np.complex128)
        counts.append(O.rsft(plan, x, estimate=False, keep=False)["votes"].reshape(-1))
    v = np.concatenate(counts)
    for mu in range(0, 4):
        emp = float(np.mean(v > mu))
        exact = O.binomial_vote_tail(loops, pfa1, mu)
        assert abs(emp / exact - 1) < 0.15, (mu, emp, exact)
    # Claim 3's Normal form with F = 0 puts the tail at mu = 4 far below the binomial law and the votes
    normal = O.q_func((4 - loops * pfa1) / math.sqrt(loops * pfa1 * (1 - pfa1)))
    assert normal < 0.05 * O.binomial_vote_tail(loops, pfa1, 4)
    assert normal < 0.05 * float(np.mean(v > 4))


def test_binomial_design_solves_its_laws():
    d = O.optimal_thresholds_binomial(12, 16384, 32, 2.34 ** 3, 0.9, 1e-6)
    mu, pd, q = d["mu"], d["pd_bar"], d["pfa1"]
    assert O.binomial_vote_tail(12, pd, mu) == pytest.approx(0.9, rel=1e-9)
    hit = min(1.0, pd)
    assert O.binomial_vote_tail(12, d["rho"] * hit + (1 - d["rho"]) * q, mu) == pytest.approx(1e-6, rel=1e-6)
    # the paper's Normal design of the same system, evaluated with the binomial law, misses P_fa by orders
    nd = O.optimal_thresholds(12, 16384, 32, 2.34 ** 3, 0.9, 1e-6)
    true_pfa = O.binomial_vote_tail(12, d["rho"] * min(1.0, nd["pd_bar"]) + (1 - d["rho"]) * nd["pfa1"], nd["mu"])
    assert true_pfa > 100 * 1e-6
    assert d["mu"] > nd["mu"]


def test_binomial_law_on_target_cubes():
    # off-target cells of cubes with targets (outside each target's +-3-bin box): with the measured
    # per-loop vote rate q, the tail of the votes is closer to Binomial(L, q) than to the Normal law
    # of the same mean and variance (Claim 3's form) at the upper thresholds a P_fa design uses.
    # It is heavier than both: a cell's collision rate with a target depends on the 2-adic
    # structure of their index difference (Def. 3), so cells differ and the mixture is overdispersed.
    n, b, loops, k = (256, 256), (16, 16), 10, 6
    bt = int(np.prod(b))
    off = []
    for seed in range(4):
        tg = ri.draw_targets(n, k, "ongrid", 40 + seed, (15.0, 15.0), bt)
        x = ri.tone_cube(n, tg, 1.0, 40 + seed).astype(np.complex128)
        plan = O.make_plan(n, b, loops, seed=200 + seed, atten_db=60.0, noise_var=1.0, pfa1=0.02, mu=0)
        votes = O.rsft(plan, x, estimate=False, keep=False)["votes"]
        near = np.zeros(n, dtype=bool)
        for gi in tg.grid_index(n):
            near[tuple(slice(max(0, int(g) - 3), int(g) + 4) for g in gi)] = True
        off.append(votes[~near])
    v = np.concatenate(off)
    q = float(v.mean()) / loops
    for mu in (3, 4, 5):
        emp = float(np.mean(v > mu))
        binom = O.binomial_vote_tail(loops, q, mu)
        normal = O.q_func((mu - loops * q) / math.sqrt(loops * q * (1 - q)))
        assert abs(math.log(emp / binom)) < abs(math.log(emp / normal)), (mu, emp, binom, normal)
        assert emp / binom < 10.0, (mu, emp, binom)
