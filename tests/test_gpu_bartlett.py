"""Parity of the dense Bartlett detector (Appendix A, Algorithm 2, one segment) with the
FP64 oracle: spectrum within 1e-4 (relative, 0.1 rms floor), detected bins bit-exact
outside a 1e-5 band around the threshold, amplitudes within 1e-4."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1610_01050_gb300 as R
import rsft_inputs as ri
from tests.gpu_helpers import BAND, REL_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1610_01050_gb300 import build as B
    B.build()
    R.load_library()


def _run(n, window, atten, nv, p_fa, cube, cap=1 << 20):
    d = R.make_desc(n, tuple(max(1, x // 8) for x in n), 4, window=window, atten_db=atten, noise_var=nv,
                    max_located=cap)
    d.p_fa = p_fa
    plan = R.rsft_bartlett_plan_create(d)
    x = torch.from_numpy(np.ascontiguousarray(cube)).cuda()
    loc = torch.zeros(max(cap, 1), dtype=torch.int64, device="cuda")
    amp = torch.zeros(max(cap, 1), dtype=torch.complex64, device="cuda")
    cnt = R.rsft_bartlett_execute(plan, x, located=loc, amp=amp, allow_capacity=True)
    spec = torch.empty(int(np.prod(n)), dtype=torch.complex64, device="cuda")
    R.rsft_bartlett_copy_spectrum(plan, spec)
    torch.cuda.synchronize()
    k = min(cnt, cap)
    return plan, cnt, loc[:k].cpu().numpy(), amp[:k].cpu().numpy(), spec.cpu().numpy().reshape(n)


def _compare(plan, cnt, loc, amp, spec, ref):
    assert abs(float(R.rsft_bartlett_get(plan, R.RSFT_BARTLETT_GAMMA)[0]) - ref["gamma"]) <= 1e-9 * ref["gamma"]
    e = rel_err(spec, ref["spectrum"])
    assert e <= REL_TOL, f"spectrum rel err {e}"
    band = np.abs(ref["power"].reshape(-1) - ref["gamma"]) <= BAND * ref["gamma"]
    keep_g = ~band[loc]
    keep_r = ~band[ref["located"]]
    np.testing.assert_array_equal(loc[keep_g], ref["located"][keep_r])
    assert np.all(np.diff(loc) > 0)
    if keep_r.any():
        ea = rel_err(amp[keep_g], ref["amplitudes"][keep_r])
        assert ea <= REL_TOL, f"amplitude rel err {ea}"
    return int(band.sum())


CASES = [
    ("2d_cheb", (256, 256), R.RSFT_WIN_CHEB, 60.0, 1e-3),
    ("3d_cheb80", (64, 32, 16), R.RSFT_WIN_CHEB, 80.0, 1e-4),
    ("1d", (4096,), R.RSFT_WIN_CHEB, 50.0, 1e-2),
    ("4d", (16, 16, 8, 8), R.RSFT_WIN_CHEB, 60.0, 1e-3),
    ("2d_rect", (128, 64), R.RSFT_WIN_RECT, 0.0, 1e-3),
]


@pytest.mark.parametrize("name,n,window,atten,p_fa", CASES, ids=[c[0] for c in CASES])
def test_bartlett_parity(name, n, window, atten, p_fa):
    seed = 900 + len(name)
    tg = ri.draw_targets(n, 6, "offgrid", seed, (10.0, 25.0), int(np.prod(n)) // 64)
    cube = ri.tone_cube(n, tg, 1.0, seed)
    plan, cnt, loc, amp, spec = _run(n, window, atten, 1.0, p_fa, cube)
    ref = O.bartlett(cube.astype(np.complex128), "cheb" if window == R.RSFT_WIN_CHEB else "rect", atten, 1.0, p_fa)
    _compare(plan, cnt, loc, amp, spec, ref)
    assert cnt == len(loc)


def test_bartlett_full_radar_cube():
    # the 3-D radar workload at full size (1024 x 256 x 64), one frame
    cube, targets, wl, nv = ri.workload_frame("c2_3d_radar", 0)
    plan, cnt, loc, amp, spec = _run(wl.shape, R.RSFT_WIN_CHEB, wl.atten_db, nv, wl.p_fa, cube)
    ref = O.bartlett(cube.astype(np.complex128), "cheb", wl.atten_db, nv, wl.p_fa)
    _compare(plan, cnt, loc, amp, spec, ref)
    assert cnt > 0


def test_bartlett_capacity_and_alignment():
    n = (64, 64)
    cube = ri.tone_cube(n, ri.draw_targets(n, 4, "ongrid", 3, (20.0, 20.0), 64), 1.0, 3)
    ref = O.bartlett(cube.astype(np.complex128), "cheb", 60.0, 1.0, 0.05)
    total = len(ref["located"])
    assert total > 4
    plan, cnt, loc, amp, spec = _run(n, R.RSFT_WIN_CHEB, 60.0, 1.0, 0.05, cube, cap=4)
    assert cnt == total
    np.testing.assert_array_equal(loc, ref["located"][:4])
    x = torch.from_numpy(cube).cuda()
    raw = torch.zeros(x.numel() * 2 + 2, dtype=torch.float32, device="cuda")
    mis = raw[1:1 + x.numel() * 2]                        # 4-byte aligned, not 16
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(R.RsftError) as ei:
        R.rsft_bartlett_execute_async(plan, mis, count)
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG
