"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and
compare it with the oracle element by element.

Tolerances (the arithmetic behind them is in the design notes):
  * folded and spectrum buckets, amplitudes: |gpu - ref| <= 1e-4 * max(|ref|, 0.1 * rms),
    rms over the loop (buckets) or over the located set (amplitudes): an FP32 sum's
    error scales with the norm of its terms, not with the value of the sum;
  * sigma tables, detections, votes and located indices: bit-exact, except buckets
    whose FP64 power lies within 1e-5 (relative) of gamma_l, which are excluded and
    reported, together with the votes and locations their candidates touch;
  * estimate mode (noise floor from the bucket powers): the GPU's threshold gamma_l is the
    oracle's within GAMMA_TOL, and within the bound the order statistic obeys (the lower
    median moves by at most the largest change of any power); the detection band then widens
    by the measured threshold difference.
"""
import numpy as np
import torch

import oracle as O
import paper_1610_01050_gb300 as R

REL_TOL = 1e-4
FLOOR = 0.1
BAND = 1e-5
GAMMA_TOL = 2.5e-4   # estimate mode: twice REL_TOL (a power's error is twice its value's)


def gpu_run(desc, cube_np=None, cube_dev=None, want_votes=True, plan=None):
    plan = plan if plan is not None else R.rsft_plan_create(desc)
    n = tuple(int(desc.n[i]) for i in range(desc.ndim))
    b = tuple(int(desc.b[i]) for i in range(desc.ndim))
    L = int(desc.loops)
    total_b = int(np.prod(b))
    cube = cube_dev if cube_dev is not None else torch.from_numpy(np.ascontiguousarray(cube_np)).cuda()
    cap = int(desc.max_located)
    dev = cube.device
    located = torch.zeros(max(cap, 1), dtype=torch.int64, device=dev)
    lvotes = torch.zeros(max(cap, 1), dtype=torch.uint8, device=dev)
    amp = torch.zeros(max(cap, 1), dtype=torch.complex64, device=dev)
    votes = torch.zeros(int(np.prod(n)), dtype=torch.uint8, device=dev) if want_votes else None
    cnt = R.rsft_execute(plan, cube, located=located, located_votes=lvotes, amp=amp, votes_out=votes,
                         allow_capacity=True)
    folded = torch.empty(L * total_b, dtype=torch.complex64, device=dev)
    spectrum = torch.empty(L * total_b, dtype=torch.complex64, device=dev)
    words = (total_b + 31) // 32
    det = torch.zeros(L * words, dtype=torch.int32, device=dev)
    R.rsft_copy_buckets(plan, R.RSFT_BUCKETS_FOLDED, folded)
    R.rsft_copy_buckets(plan, R.RSFT_BUCKETS_SPECTRUM, spectrum)
    R.rsft_copy_detections(plan, det)
    torch.cuda.synchronize()
    gamma_last = R.rsft_plan_get(plan, R.RSFT_GET_GAMMA_LAST)
    k = min(cnt, cap)
    bits = np.unpackbits(det.cpu().numpy().view(np.uint8), bitorder="little").reshape(L, words * 32)[:, :total_b]
    return {
        "plan": plan,
        "count": cnt,
        "located": located[:k].cpu().numpy().astype(np.int64),
        "located_votes": lvotes[:k].cpu().numpy(),
        "amp": amp[:k].cpu().numpy(),
        "votes": votes.cpu().numpy().reshape(n) if want_votes else None,
        "folded": folded.cpu().numpy().reshape((L,) + b),
        "spectrum": spectrum.cpu().numpy().reshape((L,) + b),
        "detected": bits.reshape((L,) + b).astype(bool),
        "gamma": gamma_last,
    }


def rel_err(gpu, ref, axis_rms=None):
    """max |gpu - ref| / max(|ref|, FLOOR * rms(ref)); rms per leading index if axis_rms."""
    ref = np.asarray(ref)
    gpu = np.asarray(gpu)
    if axis_rms is not None:
        flat = ref.reshape(ref.shape[0], -1)
        rms = np.sqrt(np.mean(np.abs(flat) ** 2, axis=1))
        rms = rms.reshape((-1,) + (1,) * (ref.ndim - 1))
    else:
        rms = np.sqrt(np.mean(np.abs(ref) ** 2)) if ref.size else 1.0
    denom = np.maximum(np.abs(ref), FLOOR * rms)
    if ref.size == 0:
        return 0.0
    return float(np.max(np.abs(gpu - ref) / denom))


def compare_tables(plan, op):
    np.testing.assert_array_equal(R.rsft_plan_get(plan, R.RSFT_GET_SIGMA), op.sigma)
    np.testing.assert_array_equal(R.rsft_plan_get(plan, R.RSFT_GET_SIGMA_INV), op.sigma_inv)
    assert int(R.rsft_plan_get(plan, R.RSFT_GET_MU)[0]) == op.mu
    np.testing.assert_allclose(R.rsft_plan_get(plan, R.RSFT_GET_GAMMA), op.gamma, rtol=1e-8)


def band_mask(op, spectrum_ref, gamma=None, rel=None):
    """Buckets whose FP64 power is within BAND (relative; per loop `rel` if given) of gamma_l."""
    power = np.abs(spectrum_ref) ** 2
    gamma = op.gamma if gamma is None else np.asarray(gamma)
    gam = gamma.reshape((-1,) + (1,) * op.ndim)
    width = BAND if rel is None else np.asarray(rel).reshape((-1,) + (1,) * op.ndim)
    return np.abs(power - gam) <= width * gam


def check_noise_floor(g, ref, op):
    """Estimate mode: the GPU's per-loop threshold against the oracle's; returns the per-loop
    relative band for the detection comparison."""
    gg, gr = np.asarray(g["gamma"], dtype=np.float64), np.asarray(ref["gamma"], dtype=np.float64)
    assert np.all(np.isfinite(gg)) and np.all(gr > 0)
    factor = float(np.float32(-np.log(op.pfa1) / np.log(2.0)))
    for l in range(op.loops):
        pg = np.abs(g["spectrum"][l].astype(np.complex128)) ** 2
        pr = np.abs(ref["spectrum"][l]) ** 2
        m_ref = gr[l] * np.log(2.0) / -np.log(op.pfa1)
        m_gpu = gg[l] / factor
        # the lower median is 1-Lipschitz in the max norm of the powers (plus FP32 rounding)
        assert abs(m_gpu - m_ref) <= np.max(np.abs(pg - pr)) + 4e-7 * m_ref, (l, m_gpu, m_ref)
    rel = np.abs(gg / gr - 1)
    assert np.all(rel <= GAMMA_TOL), rel
    # exactly: each threshold is the rank-floor((B - 1) / 2) power of the GPU's own FP32 spectrum
    # (power = fma(re, re, re(im * im)): re^2 is exact in FP64, the FP32 product im * im is rounded,
    # one final rounding to FP32) times the plan's factor, multiplied in FP32
    pfa1 = float(R.rsft_plan_get(g["plan"], R.RSFT_GET_PFA1)[0])
    f32 = np.float32(-np.log(pfa1) / np.log(2.0))
    for l in range(op.loops):
        sp = np.asarray(g["spectrum"][l]).reshape(-1)
        x, y = sp.real.astype(np.float32), sp.imag.astype(np.float32)
        pw = (x.astype(np.float64) * x.astype(np.float64) + (y * y).astype(np.float64)).astype(np.float32)
        m = np.sort(pw)[(pw.size - 1) // 2]
        assert np.float32(gg[l]) == np.float32(m) * f32, (l, gg[l], m, f32)
    return BAND + rel


def touched_by(op, band):
    """Locations whose votes a band bucket can change (its reverse-mapped candidates)."""
    mask = np.zeros(op.n, dtype=bool)
    for idx in np.argwhere(band):
        l, j = int(idx[0]), idx[1:]
        mask[np.ix_(*O.reverse_map(op, l, j))] = True
    return mask


def compare_full(g, ref, op, check_votes=True):
    """Element-wise parity of every stage; returns a small report dict."""
    compare_tables(g["plan"], op)
    e_fold = rel_err(g["folded"], ref["folded"], axis_rms=True)
    e_spec = rel_err(g["spectrum"], ref["spectrum"], axis_rms=True)
    assert e_fold <= REL_TOL, f"folded buckets rel err {e_fold}"
    assert e_spec <= REL_TOL, f"spectrum rel err {e_spec}"
    if getattr(op, "estimate_noise", False):
        band = band_mask(op, ref["spectrum"], ref["gamma"], check_noise_floor(g, ref, op))
    else:
        band = band_mask(op, ref["spectrum"])
    outside = ~band
    np.testing.assert_array_equal(g["detected"][outside], ref["detected"][outside])
    mask = touched_by(op, band) if band.any() else np.zeros(op.n, dtype=bool)
    if check_votes:
        np.testing.assert_array_equal(g["votes"][~mask], ref["votes"][~mask])
    # located sets: equal outside the cells a band bucket can touch; equal counts whenever no
    # band bucket exists (no waiver of the count, no truncation of either list)
    assert g["count"] == len(g["located"]), "located list truncated: raise max_located"
    assert np.all(np.diff(g["located"]) > 0), "located list must be strictly ascending"
    flat_mask = mask.reshape(-1)
    loc_ref = ref["located"]
    keep_ref = ~flat_mask[loc_ref]
    keep_gpu = ~flat_mask[g["located"]]
    np.testing.assert_array_equal(g["located"][keep_gpu], loc_ref[keep_ref])
    if not band.any():
        assert g["count"] == len(loc_ref), "located count differs"
    np.testing.assert_array_equal(g["located_votes"][keep_gpu], ref["located_votes"][keep_ref])
    e_amp = 0.0
    if keep_ref.any() and "amplitudes" in ref:
        e_amp = rel_err(g["amp"][keep_gpu], ref["amplitudes"][keep_ref])
        assert e_amp <= REL_TOL, f"amplitude rel err {e_amp}"
    return {"fold": e_fold, "spectrum": e_spec, "amp": e_amp, "band": int(band.sum()),
            "located": len(loc_ref), "touched": int((~keep_ref).sum()), "detected": int(ref["detected"].sum())}
