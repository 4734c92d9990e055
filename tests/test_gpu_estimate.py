"""GPU parity of the first stage's estimate mode (noise level unknown, §IV-B): each loop's
threshold is the lower median of its bucket powers divided by ln 2, times -ln Pfa1.

The CUDA path (radix select of the median over the FP32 powers, then detection) is compared
with the FP64 oracle: thresholds within GAMMA_TOL and within the order statistic's
Lipschitz bound, detections bit-exact outside a band widened by the measured threshold
difference, votes, located sets and amplitudes as in known-noise mode.  Sizes cover bucket
counts below a warp (B = 8), a ragged vote tail, every dimension count, and B = 65536, whose
powers do not fit in shared memory (the select then re-reads the spectrum per digit).
"""
import zlib

import numpy as np
import pytest
import torch

import oracle as O
import rsft_inputs as ri
import paper_1610_01050_gb300 as R
from paper_1610_01050_gb300 import build as B
from tests.gpu_helpers import gpu_run, compare_full

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    R.load_library()


CASES = [
    ("2d_256", (256, 256), (16, 16), 8, 0.02, 2),
    ("3d_rows", (64, 32, 16), (8, 4, 4), 5, 0.03, 1),
    ("1d", (4096,), (64,), 3, 0.05, 1),
    ("4d", (16, 16, 8, 8), (4, 4, 2, 2), 10, 0.05, 3),
    ("2d_b8", (64, 32), (4, 2), 6, 0.1, 2),
    ("2d_b65536", (512, 512), (256, 256), 4, 1e-3, 1),
    ("3d_radar_shape", (128, 64, 32), (16, 8, 4), 12, 0.01, 3),
]


@pytest.mark.parametrize("name,n,b,loops,pfa1,mu", CASES, ids=[c[0] for c in CASES])
def test_estimate_mode_parity(name, n, b, loops, pfa1, mu):
    seed = zlib.crc32(name.encode()) % 1000
    nv = 1.7                                      # the library is not told this
    tg = ri.draw_targets(n, 6, "offgrid", seed, (8.0, 20.0), int(np.prod(b)), noise_var=nv)
    cube = ri.tone_cube(n, tg, nv, seed)
    d = R.make_desc(n, b, loops, seed=seed, p_fa1=pfa1, mu=mu, noise_var=0.0, max_located=1 << 20)
    op = O.make_plan(n, b, loops, seed=seed, pfa1=pfa1, mu=mu, noise_var=0.0)
    g = gpu_run(d, cube)
    ref = O.rsft(op, cube.astype(np.complex128))
    rep = compare_full(g, ref, op)
    print(f"estimate {name}: {rep}, gamma rel diff {np.max(np.abs(g['gamma'] / ref['gamma'] - 1)):.2e}")
    assert rep["detected"] > 0


def test_estimate_mode_repeat_and_scale():
    """Two executes agree bit for bit; a cube scaled by 8 (exact in FP32) scales every threshold by
    64 and leaves the detections, votes and located set unchanged."""
    n, b, loops = (128, 64, 16), (16, 8, 4), 8
    tg = ri.draw_targets(n, 5, "offgrid", 3, (10.0, 20.0), int(np.prod(b)))
    cube = ri.tone_cube(n, tg, 1.0, 3)
    d = R.make_desc(n, b, loops, seed=3, p_fa1=0.02, mu=2, noise_var=-1.0)
    plan = R.rsft_plan_create(d)
    a = gpu_run(d, cube, plan=plan)
    a2 = gpu_run(d, cube, plan=plan)
    s = gpu_run(d, (8.0 * cube).astype(np.complex64), plan=plan)
    np.testing.assert_array_equal(a["gamma"], a2["gamma"])
    np.testing.assert_array_equal(a["located"], a2["located"])
    np.testing.assert_array_equal(s["gamma"], 64.0 * a["gamma"])
    np.testing.assert_array_equal(s["detected"], a["detected"])
    np.testing.assert_array_equal(s["votes"], a["votes"])
    np.testing.assert_array_equal(s["located"], a["located"])


def test_estimate_mode_noise_only_rate():
    """Noise-only radar-shaped cubes: the detection rate of the GPU's estimate mode agrees with
    the closed form for independent exponential powers (test_oracle_estimate) within 20 %."""
    from tests.test_oracle_estimate import expected_detections
    n, b, loops, pfa1 = (256, 128, 32), (32, 16, 8), 12, 1e-3
    bt = int(np.prod(b))
    d = R.make_desc(n, b, loops, seed=11, p_fa1=pfa1, mu=5, noise_var=0.0)
    plan = R.rsft_plan_create(d)
    hits = 0
    frames = 4
    for f in range(frames):
        g = gpu_run(d, ri.tone_cube(n, None, 0.3, 500 + f), plan=plan, want_votes=False)
        hits += int(g["detected"].sum())
    rate = hits / (frames * loops * bt)
    expect = expected_detections(bt, pfa1) / bt
    assert abs(rate / expect - 1) < 0.2, (rate, expect)


def test_estimate_mode_full_radar_workload():
    """The 1024 x 256 x 64 radar workload (B = 64 x 32 x 8, L = 12) in estimate mode, every stage
    against the oracle."""
    cube, tg, wl, nv = ri.workload_frame("c2_3d_radar")
    d = R.make_desc(wl.shape, wl.buckets, wl.loops, seed=ri.frame_seed(wl, 0), atten_db=wl.atten_db, p_fa=wl.p_fa,
                    k_max=wl.k_design, noise_var=0.0, max_located=1 << 20)
    op = O.make_plan(wl.shape, wl.buckets, wl.loops, seed=ri.frame_seed(wl, 0), atten_db=wl.atten_db, p_fa=wl.p_fa,
                     k_max=wl.k_design, noise_var=0.0)
    g = gpu_run(d, cube)
    ref = O.rsft(op, cube.astype(np.complex128))
    rep = compare_full(g, ref, op)
    print(f"estimate c2_3d_radar: {rep}")
    assert rep["located"] > 0
