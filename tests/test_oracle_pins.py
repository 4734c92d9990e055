"""Pins of the CPU oracle against the paper and the mathematics (no GPU).

Every check here compares the oracle with something other than itself: a
published constant, a library routine, a closed form, an identity the paper
states, a hand-derived worked example, or exhaustive brute force.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.signal.windows import chebwin
from scipy.stats import beta as beta_dist

import oracle as O
import rsft_inputs as ri

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ----------------------------------------------------------------------------- draws

def test_splitmix64_published_sequence():
    # First outputs of SplitMix64 from state 0 (Vigna's reference splitmix64.c).
    assert O.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("n", [(2,), (64, 32), (1024, 256, 64), (512, 512, 64, 32)])
def test_sigma_odd_uniform_and_invertible(n):
    sig = O.draw_sigmas(123, 40, n)
    assert sig.shape == (40, len(n))
    for d, nd in enumerate(n):
        assert np.all(sig[:, d] % 2 == 1) and np.all((0 < sig[:, d]) & (sig[:, d] < nd))
        for s in sig[:, d]:
            inv = O.inverse_mod(int(s), nd)
            assert (int(s) * inv) % nd == 1          # eq. (mod_inv)


# ----------------------------------------------------------------------------- windows

@pytest.mark.parametrize("n", [2, 3, 8, 63, 64, 255, 256, 1024])
@pytest.mark.parametrize("atten", [45.0, 60.0, 80.0])
def test_chebyshev_matches_scipy(n, atten):
    np.testing.assert_allclose(O.chebyshev_window(n, atten), chebwin(n, atten), atol=1e-11, rtol=0)


@pytest.mark.parametrize("atten", [40.0, 60.0, 80.0])
def test_chebyshev_equiripple_sidelobes(atten):
    n = 64
    w = O.chebyshev_window(n, atten)
    spec = np.abs(np.fft.fft(w, n * 256))
    spec /= spec[0]
    db = 20 * np.log10(np.maximum(spec, 1e-300))
    first_null = int(np.argmax(np.diff(db[: n * 128]) > 0))   # end of the main lobe
    side = db[first_null: n * 256 - first_null]
    peaks = side[1:-1][(side[1:-1] >= side[:-2]) & (side[1:-1] >= side[2:])]
    assert abs(np.max(peaks) + atten) < 0.02          # side lobes at -A dB ...
    assert np.all(peaks > -atten - 0.5)               # ... all of them (equiripple)


def test_chebyshev_symmetric_peak_one():
    for n in (64, 65, 1024):
        w = O.chebyshev_window(n, 60.0)
        np.testing.assert_allclose(w, w[::-1], atol=1e-14)
        assert abs(w.max() - 1.0) < 1e-15


def test_rect_window_6db_bandwidth_textbook():
    # The 6-dB bandwidth of the rectangular window is 1.21 bins (Harris 1978).
    assert abs(O.window_6db_bins(np.ones(256)) - 1.207) < 0.002
    bw = [O.window_6db_bins(O.chebyshev_window(1024, a)) for a in (40.0, 60.0, 80.0)]
    assert bw[0] < bw[1] < bw[2]                      # wider main lobe for deeper side lobes


@pytest.mark.parametrize("n,m", [(64, 8), (256, 16), (32, 1), (16, 16)])
def test_ideal_flat_window_is_boxcar(n, m):
    wbar = O.flat_window(n, m, "ideal", 60.0)
    g = O.flat_gain(wbar)
    expect = np.zeros(n)
    expect[(-np.arange(m)) % n] = 1.0                   # pass band u in (-M, 0]
    np.testing.assert_allclose(g, expect, atol=1e-12)


@pytest.mark.parametrize("n,m,support", [(256, 16, None), (1024, 16, None), (256, 16, 64)])
def test_cheb_flat_window_passband(n, m, support):
    wbar = O.flat_window(n, m, "cheb", 60.0, support)
    g = O.flat_gain(wbar)
    assert abs(g[(-(m // 2)) % n] - 1.0) < 1e-12       # normalised at mid pass band
    t = np.arange(n)
    if support is not None:                            # zero outside the support
        half = (support - 2) // 2
        outside = (t > half) & (t < n - half)
        assert np.all(wbar[outside] == 0)
    if support is None:
        mid = np.abs(g[(-np.arange(m // 4, 3 * m // 4)) % n])
        assert np.all(np.abs(mid - 1) < 0.05)          # flat pass band
        stop = np.abs(g[np.arange(4, n - m - 4)])
        assert np.max(stop) < 0.02                     # suppressed outside


# ----------------------------------------------------------------------------- identities

def _rand_cube(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("shape,sigma", [((16,), (5,)), ((16, 8), (3, 7)), ((8, 4, 16), (5, 3, 11))])
def test_permutation_property(shape, sigma):
    # Prop. 1 with tau = 0: DFT of p(t) = x(sigma t) at sigma f equals X(f).
    x = _rand_cube(shape, 1)
    X = np.fft.fftn(x)
    P = np.fft.fftn(O.permute(x, sigma))
    idx = np.indices(shape)
    perm = tuple((s * idx[d]) % shape[d] for d, s in enumerate(sigma))
    np.testing.assert_allclose(P[perm], X, atol=1e-9)


@pytest.mark.parametrize("shape,b", [((16,), (4,)), ((16, 32), (4, 8)), ((8, 16, 4), (2, 4, 1))])
def test_aliasing_property(shape, b):
    # Prop. 2: the B-point DFT of the aliased signal is the N-point DFT subsampled by M.
    z = _rand_cube(shape, 2)
    Y = np.fft.fftn(O.alias(z, b))
    Z = np.fft.fftn(z)
    m = [n // bb for n, bb in zip(shape, b)]
    np.testing.assert_allclose(Y, Z[tuple(slice(None, None, mm) for mm in m)], atol=1e-9)


def test_ideal_flat_fold_is_bucket_sum():
    # Ideal flat window: bucket k collects exactly the permuted bins [kM, (k+1)M).
    n, b = (32, 16), (4, 2)
    plan = O.make_plan(n, b, 3, seed=9, window="cheb", atten_db=60.0, flat="ideal", pfa1=0.1, mu=1)
    r = _rand_cube(n, 3)
    m = plan.m
    for l in range(plan.loops):
        fh = O.bucket_spectrum(O.fold_loop(plan, r, l))
        y = np.multiply.outer(plan.w[0], plan.w[1]) * r
        P = np.fft.fftn(O.permute(y, plan.sigma[l]))
        expect = P.reshape(b[0], m[0], b[1], m[1]).sum(axis=(1, 3))
        np.testing.assert_allclose(fh, expect, atol=1e-9)


def _dense_matrix_spectrum(plan, r, l):
    # eq. (l) and eq. (f): f-hat = D V_sigma r, V_sigma = sum_i W-bar_i P_sigma W, one
    # Kronecker factor per dimension (row-major flattening).
    V = np.ones((1, 1))
    Dm = np.ones((1, 1))
    for d in range(plan.ndim):
        n, b = plan.n[d], plan.b[d]
        perm = np.zeros((n, n))
        perm[np.arange(n), (plan.sigma[l, d] * np.arange(n)) % n] = 1.0    # (P y)_t = y_{sigma t}
        wbar_p_w = np.diag(plan.wbar[d]) @ perm @ np.diag(plan.w[d])
        alias = np.zeros((b, n))
        alias[np.arange(n) % b, np.arange(n)] = 1.0
        V = np.kron(V, alias @ wbar_p_w)
        Dm = np.kron(Dm, np.exp(-2j * np.pi * np.outer(np.arange(b), np.arange(b)) / b))
    return (Dm @ V @ r.reshape(-1)).reshape(plan.b)


@pytest.mark.parametrize("n,b,flat", [((16, 16), (4, 2), "cheb"), ((8, 16), (2, 4), "ideal"), ((32,), (8,), "cheb")])
def test_dense_matrix_form(n, b, flat):
    plan = O.make_plan(n, b, 3, seed=5, atten_db=60.0, flat=flat, pfa1=0.1, mu=1)
    r = _rand_cube(n, 4)
    for l in range(plan.loops):
        got = O.bucket_spectrum(O.fold_loop(plan, r, l))
        np.testing.assert_allclose(got, _dense_matrix_spectrum(plan, r, l), atol=1e-9)


def test_bucket_fft_brute_force_16x16():
    f = _rand_cube((16, 16), 6)
    k = np.arange(16)
    W = np.exp(-2j * np.pi * np.outer(k, k) / 16)
    brute = np.array([[np.sum(f * np.outer(W[a], W[c])) for c in range(16)] for a in range(16)])
    np.testing.assert_allclose(O.bucket_spectrum(f), brute, atol=1e-9)
    # Parseval: sum |f-hat|^2 = B sum |f|^2
    assert abs(np.sum(np.abs(brute) ** 2) - 256 * np.sum(np.abs(f) ** 2)) < 1e-8 * np.sum(np.abs(brute) ** 2)


def test_fold_bucket_direct_matches_loop():
    plan = O.make_plan((32, 16, 8), (4, 4, 2), 2, seed=2, atten_db=80.0, pfa1=0.1, mu=1)
    r = _rand_cube(plan.n, 7)
    for l in range(2):
        f = O.fold_loop(plan, r, l)
        for j in [(0, 0, 0), (3, 1, 1), (2, 3, 0)]:
            assert abs(O.fold_bucket_direct(plan, r, l, j) - f[j]) < 1e-10


def test_worked_example_4x8():
    # Fig. Permutation: x[i, j] = 8 i + j, sigma_x = sigma_y = 3, tau = 0, B = 2 x 4.
    x = np.arange(32, dtype=np.float64).reshape(4, 8)
    p = O.permute(x, (3, 3))
    expect_p = np.array([[0, 3, 6, 1, 4, 7, 2, 5],
                         [24, 27, 30, 25, 28, 31, 26, 29],
                         [16, 19, 22, 17, 20, 23, 18, 21],
                         [8, 11, 14, 9, 12, 15, 10, 13]], dtype=np.float64)
    np.testing.assert_array_equal(p, expect_p)
    expect_f = np.array([[40, 52, 48, 44], [72, 84, 80, 76]], dtype=np.float64)
    np.testing.assert_array_equal(O.alias(p, (2, 4)), expect_f)


@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_reversibility_and_distinctiveness_exhaustive(n):
    # Prop. 3 (i in R(M(i, sigma), sigma^{-1})) and Prop. 4 (R(j) disjoint), App. B.
    for b in [bb for bb in (1, 2, 4, 8, 16, 32, 64) if bb <= n]:
        m = n // b
        for s in range(1, n, 2):
            plan = O.OraclePlan(n=(n,), b=(b,), m=(m,), loops=1, sigma=np.array([[s]]),
                                sigma_inv=np.array([[O.inverse_mod(s, n)]]), w=[], wbar=[],
                                gain=[], wsum=1.0, beta=np.ones(1), gamma=np.ones(1), mu=0,
                                pfa1=0.1, noise_var=1.0, eta_m=1.0)
            cover = np.zeros(n, dtype=int)
            for j in range(b):
                rj = O.reverse_map(plan, 0, (j,))[0]
                assert len(set(rj.tolist())) == m
                cover[rj] += 1
                for i in rj:
                    assert O.mapping(plan, 0, (int(i),)) == (j,)
            assert np.all(cover == 1)                      # a partition of [N]


# ----------------------------------------------------------------------------- end to end

def _exact_case(n, b, loops, k, seed):
    tg = ri.draw_targets(n, k, "ongrid", seed, (0, 0), int(np.prod(b)), amp_model="rayleigh")
    idx = np.indices(n)
    x = sum(a * np.exp(2j * np.pi * sum(f[d] * idx[d] for d in range(len(n))))
            for f, a in zip(tg.freqs, tg.amps))
    return x, tg


@pytest.mark.parametrize("n,b,loops,k", [((64, 32), (8, 8), 6, 4), ((32, 16, 8), (4, 4, 2), 5, 3),
                                         ((256,), (16,), 7, 3),
                                         ((32, 16), (4, 4), 255, 2)])   # the largest L: 255 votes, mu = 254
def test_exact_recovery_noise_free(n, b, loops, k):
    x, tg = _exact_case(n, b, loops, k, 17)
    tiny = 1e-6 * np.min(np.abs(tg.amps)) ** 2
    plan = O.make_plan(n, b, loops, seed=4, window="rect", flat="ideal",
                       pfa1=math.exp(-1.0), mu=loops - 1, noise_var=tiny)
    out = O.rsft(plan, x)
    truth = np.ravel_multi_index(tg.grid_index(n).T, n)
    grid = tg.grid_index(n)
    # detected buckets are exactly the mapped truth, loop by loop (Def. 3, Claim 1)
    for l in range(loops):
        expect = np.zeros(plan.b, dtype=bool)
        for g in grid:
            expect[O.mapping(plan, l, g)] = True
        np.testing.assert_array_equal(out["detected"][l], expect)
    votes = out["votes"].reshape(-1)
    assert np.all(votes[truth] == loops)
    # brute force: a location reaches L votes iff it shares a bucket with a tone in every loop
    allv = np.ones(int(np.prod(n)), dtype=bool)
    for l in range(loops):
        occ = {O.mapping(plan, l, g) for g in grid}
        per = np.array([O.mapping(plan, l, np.unravel_index(i, n)) in occ for i in range(int(np.prod(n)))])
        allv &= per
    np.testing.assert_array_equal(out["located"], np.flatnonzero(allv))
    # amplitudes are exact where the tone is alone in its bucket in a majority of loops
    order = np.argsort(truth)
    for q, i in enumerate(np.sort(truth)):
        pos = int(np.searchsorted(out["located"], i))
        assert abs(out["amplitudes"][pos] - tg.amps[order][q]) < 1e-12 * max(1.0, abs(tg.amps[order][q]))


def test_noise_only_power_is_exponential():
    # §IV-B: under H0 the bucket power is exponential with mean sigma_n^2 beta(sigma)
    # (eq. (exp), eq. (var_fu)), so the per-bucket false-alarm rate at gamma_l is Pfa1.
    n, b, loops, nv, pfa1 = (64, 128), (16, 16), 16, 2.5, 0.05
    plan = O.make_plan(n, b, loops, seed=31, atten_db=60.0, noise_var=nv, pfa1=pfa1, mu=3)
    ratios, hits, total = [], 0, 0
    for frame in range(8):
        x = ri.tone_cube(n, None, nv, 5000 + frame).astype(np.complex128)
        out = O.rsft(plan, x, estimate=False, keep=False)
        for l in range(loops):
            pw = np.abs(out["spectrum"][l]) ** 2
            ratios.append(pw.reshape(-1) / (nv * plan.beta[l]))
            hits += int(out["detected"][l].sum())
            total += pw.size
    ratios = np.concatenate(ratios)
    se = 1.0 / math.sqrt(len(ratios))
    assert abs(ratios.mean() - 1.0) < 5 * se           # exponential mean
    assert abs(np.mean(ratios > math.log(2)) - 0.5) < 5 * 0.5 * se   # median = mean ln 2
    lo = beta_dist.ppf(0.0005, hits, total - hits + 1)
    hi = beta_dist.ppf(0.9995, hits + 1, total - hits)
    assert lo <= pfa1 <= hi                            # 99.9 % Clopper-Pearson


# ----------------------------------------------------------------------------- design

def test_complexity_optima_fig6():
    g = GOLDEN["complexity_optimum"]
    for k, best in g["k_to_best_b"].items():
        costs = [O.complexity_rsft(g["n"], b, g["loops"], int(k), g["eta_m"], g["eta_p"]) for b in g["b_grid"]]
        assert g["b_grid"][int(np.argmin(costs))] == best
    assert O.complexity_rsft(1024, 1024, 50, 5, 1.4) > O.complexity_bartlett(1024, 50) * 0.5


def _fig_design(eta_p):
    g = GOLDEN["threshold_lower_bound"]
    n, b = g["n"], g["b"]
    w = O.chebyshev_window(n, g["atten_db"])
    wb = O.flat_window(n, n // b, "cheb", g["atten_db"])
    ab = O.mean_alpha([wb], [w], [b], [2 * math.pi * g["tone_bin"] / n])
    bb = O.mean_beta([wb], [w])
    d = O.optimal_thresholds(g["loops"], b, g["k"], g["eta_m"], g["p_d"], g["p_fa"], eta_p, ab, bb)
    return d, bb, g


def test_design_lower_bound_fig8():
    d, bb, g = _fig_design(1.0)
    assert abs(d["snr_db"] - g["snr_min_db"]) < 1.0
    assert abs(d["mu"] / g["loops"] - g["mu_over_t"]) < 0.06
    # the paper normalises gamma by N^2 (an FFT scaled by 1/N): gamma* within 10 %
    gamma = O.first_stage_gamma(1.0, bb, d["pfa1"]) / g["n"] ** 2
    assert abs(gamma / g["gamma"] - 1.0) < 0.10


def test_design_upper_bound_fig9():
    d, bb, _ = _fig_design("upper")
    up = GOLDEN["threshold_upper_bound"]
    lo, _, g = _fig_design(1.0)
    assert abs(d["snr_db"] - up["snr_min_db"]) < 1.0
    assert d["snr_db"] > lo["snr_db"] and d["mu"] > lo["mu"]        # Remark 1 direction
    gamma = O.first_stage_gamma(1.0, bb, d["pfa1"]) / g["n"] ** 2
    assert abs(gamma / up["gamma"] - 1.0) < 0.10


def test_design_equations_hold_at_optimum():
    d = O.optimal_thresholds(12, 16384, 32, 12.5, 0.9, 1e-6)
    mu, pd, q, f = d["mu"], d["pd_bar"], d["pfa1"], d["f_count"]
    assert abs(O.q_func((mu - 12 * pd) / math.sqrt(12 * pd * (1 - pd))) - 0.9) < 1e-9
    mean = f * pd + (12 - f) * q
    sd = math.sqrt(f * pd * (1 - pd) + (12 - f) * q * (1 - q))
    assert abs(O.q_func((mu - mean) / sd) / 1e-6 - 1.0) < 1e-6
    for row in d["table"]:
        assert row[3] >= d["snr"] - 1e-15              # the minimiser over mu in [L]
