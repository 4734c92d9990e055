"""Algorithm 1 (RSFT) and the estimation step, literally, in FP64 (oracle side).

Notation: D dimensions of sizes N_d (powers of two, §II-A notation), bucket
grid B_d dividing N_d, fold factor M_d = N_d / B_d (the paper's L of Def. 2),
loops l in [L] (the paper's T of Algorithm 1, §IV-A).  The cube is indexed
row-major, last dimension fastest.  Per loop (Algorithm 1):

    y = W r                      pre-permutation window (§III-A, §III-C.1)
    p = P_{sigma,0} y            p(t) = y(sigma t mod N), per dimension (Def. 1, §III-C.2)
    z = W-bar p                  flat window (§IV-B)
    f = Aliasing(z)              f[j] = sum_m z[j + B m], per dimension (Def. 2, §III-C.3)
    f-hat = NDFFT(f)             forward, unnormalised (eq. (f), eq. (f_k))
    c = |f-hat|^2 > gamma_l      first-stage detection (§IV-B, eq. (tpd))
    a = Reverse(c)               R(j, sigma^{-1}) per dimension, Cartesian product (Def. 4, §III-C.4)
    votes += a                   accumulation (eq. (a_i), §III-C.5)

then o = {i : votes[i] > mu} (second-stage detection, §III-C.5), and for each
i in o the amplitude is the component-wise median over loops of
f-hat_l[M(i, sigma_l)] divided by the flat-window gain and the pre-window's
DC gain (the estimation paragraph of §III, before Algorithm 1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .perm import draw_sigmas, inverse_mod
from .windows import pre_window, flat_window, flat_gain, window_6db_bins
from .design import beta_sigma, optimal_thresholds, optimal_thresholds_binomial, first_stage_gamma


@dataclasses.dataclass
class OraclePlan:
    n: tuple
    b: tuple
    m: tuple
    loops: int
    sigma: np.ndarray        # [L, D] odd
    sigma_inv: np.ndarray    # [L, D]
    w: list                  # pre-window taps per dimension (real)
    wbar: list               # flat-window taps per dimension (complex)
    gain: list               # G_d(u) = DFT(w-bar_d)[u] / N_d
    wsum: float              # prod_d sum_t w_d(t): DC gain of the pre-window
    beta: np.ndarray         # [L] beta(sigma_l)
    gamma: np.ndarray        # [L] first-stage thresholds (known noise); NaN in estimate mode
    mu: int
    pfa1: float
    noise_var: float
    eta_m: float
    design: dict | None = None

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def estimate_noise(self) -> bool:
        """Estimate mode: the noise floor of each loop is taken from its own bucket powers."""
        return not self.noise_var > 0


def make_plan(n, b, loops: int, seed: int = 0, window: str = "cheb",
              atten_db: float = 60.0, flat: str = "cheb", flat_support=None,
              noise_var: float = 1.0, p_fa: float = 1e-6, p_d: float = 0.9,
              k_max: int = 8, eta_p=1.0, pfa1: float | None = None,
              mu: int | None = None, sigma=None, beta_mode: str = "exact",
              design_mode: str = "normal") -> OraclePlan:
    """Build the oracle's plan: sigma draws, windows, and both thresholds.

    ``noise_var <= 0`` selects the estimate mode of the first stage (the noise floor is
    estimated per loop from the bucket powers, ``noise_floor_gamma``); the thresholds are then
    formed at run time and ``gamma`` holds NaN.  ``design_mode`` picks the second-stage vote
    model of the threshold design: "normal" (Claims 2-3, the paper) or "binomial" (the exact
    binomial vote law, ``design.optimal_thresholds_binomial``)."""
    n = tuple(int(x) for x in n)
    b = tuple(int(x) for x in b)
    d = len(n)
    for nd, bd in zip(n, b):
        if nd < 2 or nd & (nd - 1) or bd < 1 or bd & (bd - 1) or nd % bd:
            raise ValueError("sizes must be powers of two with B_d | N_d")
    m = tuple(nd // bd for nd, bd in zip(n, b))
    if sigma is None:
        sigma = draw_sigmas(seed, loops, n)
    sigma = np.asarray(sigma, dtype=np.int64).reshape(loops, d)
    sigma_inv = np.array([[inverse_mod(sigma[l, dd], n[dd]) for dd in range(d)]
                          for l in range(loops)], dtype=np.int64)
    w = [pre_window(n[dd], window, atten_db) for dd in range(d)]
    sup = [None] * d if flat_support is None else list(flat_support)
    wbar = [flat_window(n[dd], m[dd], flat, atten_db, sup[dd]) for dd in range(d)]
    gain = [flat_gain(x) for x in wbar]
    wsum = float(np.prod([np.sum(x) for x in w]))
    beta = np.array([beta_sigma(wbar, w, sigma[l]) for l in range(loops)])
    eta_m = float(np.prod([window_6db_bins(x) for x in w]))
    design = None
    if pfa1 is None or mu is None:
        if design_mode == "binomial":
            design = optimal_thresholds_binomial(loops, int(np.prod(b)), k_max, eta_m, p_d, p_fa, eta_p)
        elif design_mode == "normal":
            design = optimal_thresholds(loops, int(np.prod(b)), k_max, eta_m, p_d, p_fa, eta_p)
        else:
            raise ValueError("design_mode must be 'normal' or 'binomial'")
        pfa1 = design["pfa1"] if pfa1 is None else pfa1
        mu = design["mu"] if mu is None else mu
    if not noise_var > 0:
        gamma = np.full(loops, np.nan)       # estimate mode: formed per loop from the data
    elif beta_mode == "mean":
        from .design import mean_beta
        bb = mean_beta(wbar, w)
        gamma = np.full(loops, first_stage_gamma(noise_var, bb, pfa1))
    else:
        gamma = np.array([first_stage_gamma(noise_var, bt, pfa1) for bt in beta])
    return OraclePlan(n=n, b=b, m=m, loops=loops, sigma=sigma, sigma_inv=sigma_inv,
                      w=w, wbar=wbar, gain=gain, wsum=wsum, beta=beta, gamma=gamma,
                      mu=int(mu), pfa1=float(pfa1), noise_var=float(noise_var),
                      eta_m=eta_m, design=design)


def _outer(vectors) -> np.ndarray:
    out = np.asarray(vectors[0])
    for v in vectors[1:]:
        out = np.multiply.outer(out, np.asarray(v))
    return out


def permute(y: np.ndarray, sigma_row) -> np.ndarray:
    """p(t) = y(sigma t mod N), each dimension on its own (Def. 1 with tau = 0, §III-C.2)."""
    idx = [(int(s) * np.arange(nd)) % nd for s, nd in zip(sigma_row, y.shape)]
    return y[np.ix_(*idx)]


def alias(z: np.ndarray, b) -> np.ndarray:
    """f[j] = sum_m z[j + B m] in every dimension (Def. 2, §III-C.3)."""
    shape = []
    for nd, bd in zip(z.shape, b):
        shape += [nd // bd, bd]
    axes = tuple(range(0, 2 * z.ndim, 2))
    return z.reshape(shape).sum(axis=axes)


def fold_loop(plan: OraclePlan, r: np.ndarray, l: int) -> np.ndarray:
    """Lines 'pre-window' to 'aliasing' of Algorithm 1 for loop l: returns f (B-shaped)."""
    r = np.asarray(r).astype(np.complex128)
    y = _outer(plan.w) * r
    p = permute(y, plan.sigma[l])
    z = _outer(plan.wbar) * p
    return alias(z, plan.b)


def bucket_spectrum(f: np.ndarray) -> np.ndarray:
    """f-hat = D f, the unnormalised forward N-D DFT of the buckets (eq. (f))."""
    return np.fft.fftn(f)


def fold_bucket_direct(plan: OraclePlan, r: np.ndarray, l: int, j) -> complex:
    """One bucket of eq. (l): f_j = sum_m w-bar(j + B m) w(sigma (j + B m)) r(sigma (j + B m))."""
    ts, ss, wb, wp = [], [], [], []
    for dd in range(plan.ndim):
        t = int(j[dd]) + plan.b[dd] * np.arange(plan.m[dd])
        s = (int(plan.sigma[l, dd]) * t) % plan.n[dd]
        ts.append(t)
        ss.append(s)
        wb.append(plan.wbar[dd][t])
        wp.append(plan.w[dd][s])
    vals = np.asarray(r)[np.ix_(*ss)].astype(np.complex128)
    return complex(np.sum(_outer(wb) * _outer(wp) * vals))


def noise_floor_gamma(power: np.ndarray, pfa1: float) -> float:
    """First-stage threshold of one loop from its own bucket powers (estimate mode).

    Under H0 a bucket's power is exponential with mean sigma_n^2 beta (eq. (exp)), whose median
    is the mean times ln 2; so the lower median of the loop's B powers (rank floor((B - 1) / 2)
    in ascending order) divided by ln 2 estimates the mean, and the threshold is that estimate
    in place of sigma_n^2 beta in gamma = -sigma_n^2 beta ln Pfa1 (eq. (tpd))."""
    flat = np.sort(np.asarray(power, dtype=np.float64).reshape(-1))
    m_hat = flat[(flat.size - 1) // 2] / math.log(2.0)
    return -m_hat * math.log(pfa1)


def spectrum_at(plan: OraclePlan, r: np.ndarray, pairs, rows_per_chunk: int = 0) -> np.ndarray:
    """f-hat_l[k] for a list of (l, k) pairs, without forming any other bucket.

    Eq. (l) followed by the bucket DFT (eq. (f)) is one sum over the cube:
        f-hat_l[k] = sum_t w-bar(t) w(sigma_l t) r(sigma_l t) e^{-j 2 pi sum_d t_d k_d / B_d},
    and with s = sigma_l t (t = sigma_l^{-1} s mod N, a bijection, Def. 1) every factor but r
    splits over the dimensions:
        f-hat_l[k] = sum_s r(s) prod_d v_d(s_d),
        v_d(s_d) = w-bar_d(t_d) w_d(s_d) e^{-j 2 pi t_d k_d / B_d},  t_d = sigma_{l,d}^{-1} s_d mod N_d.
    The cube is contracted with the pairs' vectors one dimension at a time, last dimension first,
    in slabs of the first dimension (FP64; the cube is read once for all pairs)."""
    r = np.asarray(r)
    if tuple(r.shape) != plan.n:
        raise ValueError("cube shape does not match the plan")
    pairs = [(int(l), tuple(int(x) for x in k)) for l, k in pairs]
    P = len(pairs)
    D = plan.ndim
    vecs = []
    for dd in range(D):
        n, bd = plan.n[dd], plan.b[dd]
        s = np.arange(n)
        v = np.empty((n, P), dtype=np.complex128)
        for p, (l, k) in enumerate(pairs):
            t = (int(plan.sigma_inv[l, dd]) * s) % n
            v[:, p] = plan.wbar[dd][t] * plan.w[dd][s] * np.exp(-2j * np.pi * ((t * k[dd]) % bd) / bd)
        vecs.append(v)
    out = np.zeros(P, dtype=np.complex128)
    inner = int(np.prod(plan.n[1:])) if D > 1 else 1
    step = rows_per_chunk or max(1, (1 << 22) // max(inner, 1))
    for a0 in range(0, plan.n[0], step):
        a1 = min(plan.n[0], a0 + step)
        x = r[a0:a1].astype(np.complex128)
        if D == 1:
            out += x @ vecs[0][a0:a1]
            continue
        y = x.reshape(-1, plan.n[-1]) @ vecs[-1]                     # [rows..., P]
        for dd in range(D - 2, 0, -1):                               # middle dimensions
            y = y.reshape(-1, plan.n[dd], P)
            y = np.einsum("xsp,sp->xp", y, vecs[dd])
        y = y.reshape(a1 - a0, P)
        out += np.einsum("sp,sp->p", y, vecs[0][a0:a1])
    return out


def reverse_map(plan: OraclePlan, l: int, j) -> list:
    """R(j, sigma^{-1}) per dimension: {sigma^{-1} u mod N : jM <= u < (j+1)M} (Def. 4)."""
    out = []
    for dd in range(plan.ndim):
        u = int(j[dd]) * plan.m[dd] + np.arange(plan.m[dd])
        out.append((int(plan.sigma_inv[l, dd]) * u) % plan.n[dd])
    return out


def mapping(plan: OraclePlan, l: int, i) -> tuple:
    """M(i, sigma) = floor(B/N [i sigma]_N) per dimension (Def. 3)."""
    return tuple(((int(plan.sigma[l, dd]) * int(i[dd])) % plan.n[dd]) // plan.m[dd]
                 for dd in range(plan.ndim))


def estimate_amplitudes(plan: OraclePlan, spectra: np.ndarray, located: np.ndarray) -> np.ndarray:
    """Median estimate over loops of f-hat_l[M(i, sigma_l)] / (G gain * pre-window DC gain)."""
    out = np.zeros(len(located), dtype=np.complex128)
    for q, lin in enumerate(located):
        i = np.unravel_index(int(lin), plan.n)
        vals = np.zeros(plan.loops, dtype=np.complex128)
        for l in range(plan.loops):
            k = mapping(plan, l, i)
            g = 1.0 + 0.0j
            for dd in range(plan.ndim):
                u = (k[dd] * plan.m[dd] - int(plan.sigma[l, dd]) * int(i[dd])) % plan.n[dd]
                g *= plan.gain[dd][u]
            vals[l] = spectra[l][k] / (g * plan.wsum)
        out[q] = np.median(vals.real) + 1j * np.median(vals.imag)
    return out


def rsft(plan: OraclePlan, r, estimate: bool = True, keep: bool = True) -> dict:
    """Run Algorithm 1 on cube r, then second-stage detection and estimation.

    ``r`` is one cube (every loop re-permutes the same data) or a list of L cubes, one
    segment per loop (§III-C: each iteration may process its own data segment r_s of the
    signal model of §IV-A, with sigma_s drawn per segment).
    """
    segments = isinstance(r, (list, tuple))
    if segments:
        if len(r) != plan.loops or any(tuple(np.shape(x)) != plan.n for x in r):
            raise ValueError("segment mode needs one cube of the plan's shape per loop")
    elif tuple(r.shape) != plan.n:
        raise ValueError("cube shape does not match the plan")
    votes = np.zeros(plan.n, dtype=np.int64)
    folded, spectra, detected, gammas = [], [], [], []
    for l in range(plan.loops):
        f = fold_loop(plan, r[l] if segments else r, l)
        fh = bucket_spectrum(f)
        power = np.abs(fh) ** 2
        gam = noise_floor_gamma(power, plan.pfa1) if plan.estimate_noise else plan.gamma[l]
        gammas.append(gam)
        c = power > gam
        for j in np.argwhere(c):
            votes[np.ix_(*reverse_map(plan, l, j))] += 1
        if keep:
            folded.append(f)
        spectra.append(fh)
        detected.append(c)
    located = np.flatnonzero(votes.reshape(-1) > plan.mu)
    out = {
        "votes": votes,
        "located": located,
        "located_votes": votes.reshape(-1)[located],
        "spectrum": np.stack(spectra),
        "detected": np.stack(detected),
        "gamma": np.asarray(gammas, dtype=np.float64),
    }
    if keep:
        out["folded"] = np.stack(folded)
    if estimate:
        out["amplitudes"] = estimate_amplitudes(plan, out["spectrum"], located)
    return out
