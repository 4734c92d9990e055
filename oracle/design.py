"""Threshold design and operation counts (oracle side, FP64).

First stage (§IV-B): under H0 a bucket's spectrum is CN(0, sigma_n^2 beta(sigma)),
so its power is exponential and the per-bucket false-alarm rate for threshold
gamma is exp(-gamma / (sigma_n^2 beta(sigma))) (eq. (tpd)).  The threshold used
per loop is therefore gamma_l = -sigma_n^2 beta(sigma_l) ln Pfa1 (exact
per-loop beta; eq. (bpd) averages it over sigma, kept as an option).

Second stage (§IV-C): votes are asymptotically Normal under both hypotheses
(Claims 2 and 3, upper-bound variances); eq. (opt) enumerates mu in [L],
solves P_d and P_fa for (Pd-bar, Pfa1-bar), and keeps the mu with the smallest
SNR_min = (beta-bar / alpha-bar) (ln Pfa1-bar / ln Pd-bar - 1), which follows
from eq. (bpd).

Binomial design (a reading beyond the paper, kept as an option; the paper's Normal form is
the default): sigma_l is drawn independently per loop (Def. 1), so the per-loop votes of one
cell are independent Bernoulli trials.  A true cell votes with probability Pd-bar, so its
count is Binomial(L, Pd-bar) exactly (the law Claim 2 approximates).  An off-target cell, in
each loop independently, shares its bucket with a target's main lobe with probability
rho = K eta_m / B (Claim 3's F / L) and then votes with probability min(1, eta_p Pd-bar), and
otherwise votes with probability Pfa1-bar; its count is Binomial(L, q), q = rho min(1,
eta_p Pd-bar) + (1 - rho) Pfa1-bar.  Claim 3's Normal approximation of the same count is thin
in the upper tail when q is small, which is where P_fa lives.

Operation counts: eq. (RSFT_complexity) with B log2 B for the FFT term, and the
Bartlett count of Table I.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.stats import binom, norm


def beta_sigma(wbars, ws, sigma_row) -> float:
    """beta(sigma) = || W-bar P_sigma w ||^2 (eq. (alpha_beta)), per-dimension product."""
    out = 1.0
    for wbar, w, s in zip(wbars, ws, sigma_row):
        n = len(w)
        t = np.arange(n)
        out *= float(np.sum(np.abs(wbar) ** 2 * w[(int(s) * t) % n] ** 2))
    return out


def mean_beta(wbars, ws) -> float:
    """beta-bar = E_sigma beta(sigma), sigma_d independent and uniform over odd [N_d]."""
    out = 1.0
    for wbar, w in zip(wbars, ws):
        n = len(w)
        vals = [beta_sigma([wbar], [w], [s]) for s in range(1, n, 2)]
        out *= float(np.mean(vals))
    return out


def alpha_sigma(wbar, w, b: int, sigma: int, omega: float) -> float:
    """alpha(p, sigma, omega) = |u_p^H V_sigma v(omega)|^2 for one dimension (eq. (alpha_beta)).

    V_sigma = sum_i W-bar_i P_sigma W (eq. (l)); v(omega)_s = e^{j omega s} (eq.
    (sinusoid)); p is the peak bucket of Claim 1, p = floor(B/N [sigma floor(omega / dw_N)]_N).
    """
    n = len(w)
    t = np.arange(n)
    s = (int(sigma) * t) % n
    f = (wbar * w[s] * np.exp(1j * omega * s))
    folded = f.reshape(n // b, b).sum(axis=0)
    k0 = int(math.floor(omega / (2 * math.pi / n)))
    p = ((int(sigma) * k0) % n) * b // n
    u = np.exp(2j * np.pi * p * np.arange(b) / b)
    return float(np.abs(np.vdot(u, folded)) ** 2)


def mean_alpha(wbars, ws, bs, omegas) -> float:
    """alpha-bar = E_sigma alpha (product over dimensions of independent sigma_d)."""
    out = 1.0
    for wbar, w, b, om in zip(wbars, ws, bs, omegas):
        n = len(w)
        vals = [alpha_sigma(wbar, w, b, s, om) for s in range(1, n, 2)]
        out *= float(np.mean(vals))
    return out


def q_func(x):
    """Gaussian tail Q(x) = 1 - Phi(x)."""
    return norm.sf(x)


def _bisect(fun, lo: float, hi: float, iters: int = 200) -> float:
    flo = fun(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = fun(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def solve_pd_bar(mu: int, loops: int, p_d: float):
    """Pd-bar with P_d = Q((mu - L Pd)/sqrt(L Pd (1 - Pd))) (Claim 2, eq. (opt)); None if none."""
    def fun(p):
        sd = math.sqrt(loops * p * (1 - p))
        return q_func((mu - loops * p) / sd) - p_d
    lo, hi = 1e-15, 1 - 1e-15
    if (fun(lo) > 0) == (fun(hi) > 0):
        return None
    return _bisect(fun, lo, hi)


def solve_pfa1(mu: int, loops: int, p_fa: float, f_count: float, eta_p, pd_bar: float):
    """Pfa1-bar with P_fa = Q((mu - mu_a0)/sigma_a0) (Claim 3, eq. (opt)); None if none.

    mu_a0 = F eta_p Pd + (L - F) Pfa, sigma_a0^2 = F eta_p Pd (1 - eta_p Pd)
    + (L - F) Pfa (1 - Pfa).  eta_p = "upper" means eta_p = 1 / Pd-bar
    (co-existing tones always detected, Remark 3).
    """
    ep = (1.0 / pd_bar) if eta_p == "upper" else float(eta_p)
    hit = min(1.0, ep * pd_bar)

    def fun(q):
        mean = f_count * hit + (loops - f_count) * q
        var = f_count * hit * (1 - hit) + (loops - f_count) * q * (1 - q)
        return q_func((mu - mean) / math.sqrt(var)) - p_fa
    lo, hi = 1e-300, 1 - 1e-12
    if (fun(lo) > 0) == (fun(hi) > 0):
        return None
    return _bisect(fun, lo, hi, iters=400)


def optimal_thresholds(loops: int, b: int, k: int, eta_m: float, p_d: float,
                       p_fa: float, eta_p=1.0, alpha_bar: float = 1.0,
                       beta_bar: float = 1.0) -> dict:
    """Solve eq. (opt) by enumerating mu in [L]; returns the minimiser and the table."""
    f_count = loops * k * eta_m / b
    if f_count >= loops:
        # Remark 2: K eta_m >= B makes the vote statistics of both hypotheses coincide
        raise ValueError("infeasible design: K eta_m >= B (Remark 2)")
    rows = []
    for mu in range(loops):
        pd = solve_pd_bar(mu, loops, p_d)
        if pd is None:
            continue
        q = solve_pfa1(mu, loops, p_fa, f_count, eta_p, pd)
        if q is None or q >= pd:
            continue
        snr = (beta_bar / alpha_bar) * (math.log(q) / math.log(pd) - 1.0)
        rows.append((mu, pd, q, snr))
    if not rows:
        raise ValueError("no feasible second-stage threshold")
    best = min(rows, key=lambda r: r[3])
    return {"mu": best[0], "pd_bar": best[1], "pfa1": best[2], "snr": best[3],
            "snr_db": 10 * math.log10(best[3]) if best[3] > 0 else float("-inf"),
            "f_count": f_count, "table": rows}


def binomial_vote_tail(loops: int, p: float, mu: int) -> float:
    """P(V > mu) for V ~ Binomial(L, p): the vote count of a cell whose per-loop vote
    probability is p, the loops being independent."""
    return float(binom.sf(mu, loops, p))


def solve_pd_bar_binomial(mu: int, loops: int, p_d: float):
    """Pd-bar with P(Binomial(L, Pd-bar) > mu) = P_d (the exact law behind Claim 2); None if none."""
    def fun(p):
        return binomial_vote_tail(loops, p, mu) - p_d
    lo, hi = 1e-15, 1 - 1e-15
    if (fun(lo) > 0) == (fun(hi) > 0):
        return None
    return _bisect(fun, lo, hi)


def solve_pfa1_binomial(mu: int, loops: int, p_fa: float, rho: float, eta_p, pd_bar: float):
    """Pfa1-bar with P(Binomial(L, q) > mu) = P_fa, q = rho hit + (1 - rho) Pfa1-bar (the exact
    law behind Claim 3); None when even Pfa1-bar = 0 gives a tail above P_fa."""
    ep = (1.0 / pd_bar) if eta_p == "upper" else float(eta_p)
    hit = min(1.0, ep * pd_bar)
    base = rho * hit

    def fun(q):
        return binomial_vote_tail(loops, base + (1.0 - rho) * q, mu) - p_fa
    lo, hi = 1e-300, 1 - 1e-12
    if fun(0.0) >= 0 or (fun(lo) > 0) == (fun(hi) > 0):
        return None
    return _bisect(fun, lo, hi, iters=400)


def optimal_thresholds_binomial(loops: int, b: int, k: int, eta_m: float, p_d: float,
                                p_fa: float, eta_p=1.0, alpha_bar: float = 1.0,
                                beta_bar: float = 1.0) -> dict:
    """Eq. (opt) with the binomial vote laws in place of Claims 2-3's Normal forms: enumerate
    mu in [L], solve both laws for (Pd-bar, Pfa1-bar), keep the smallest SNR_min."""
    rho = k * eta_m / b
    if rho >= 1.0:
        raise ValueError("infeasible design: K eta_m >= B (Remark 2)")
    rows = []
    for mu in range(loops):
        pd = solve_pd_bar_binomial(mu, loops, p_d)
        if pd is None:
            continue
        q = solve_pfa1_binomial(mu, loops, p_fa, rho, eta_p, pd)
        if q is None or q >= pd:
            continue
        snr = (beta_bar / alpha_bar) * (math.log(q) / math.log(pd) - 1.0)
        rows.append((mu, pd, q, snr))
    if not rows:
        raise ValueError("no feasible second-stage threshold")
    best = min(rows, key=lambda r: r[3])
    return {"mu": best[0], "pd_bar": best[1], "pfa1": best[2], "snr": best[3],
            "snr_db": 10 * math.log10(best[3]) if best[3] > 0 else float("-inf"),
            "rho": rho, "f_count": loops * rho, "table": rows}


def first_stage_gamma(noise_var: float, beta: float, pfa1: float) -> float:
    """gamma = -sigma_n^2 beta ln Pfa1 (inverse of eq. (tpd))."""
    return -noise_var * beta * math.log(pfa1)


def complexity_rsft(n: int, b: int, loops: int, k: int, eta_m: float, eta_p: float = 1.0) -> float:
    """Eq. (RSFT_complexity) with B log2 B for the FFT term (reproduces the optima of §IV-D)."""
    return loops * (n + b + b * math.log2(b) + k * eta_m * n / (b * eta_p)) + n


def complexity_bartlett(n: int, loops: int) -> float:
    """Table I total: T N (1 + log2 N) + N."""
    return loops * n * (1 + math.log2(n)) + n
