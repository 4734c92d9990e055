"""Frames of one plan in one launch per stage (rsft_execute_frames): the persistent fold runs
over (frame, unit), the cluster FFT, detection, vote count, second stage and median take every
frame's loops in one launch.  Each frame's located list, count and amplitudes must equal those of
a single rsft_execute of the same cube (the same kernels, the same reduction order), over group
boundaries (16 frames per launch), in estimate mode, recorded as a CUDA graph, and for plans whose
stages run the frames one after another; one frame is also checked against the oracle."""
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


CAP = 1 << 14


def _cubes(n, b, count, k=6, nv=1.0, seed0=300):
    out = []
    for f in range(count):
        tg = ri.draw_targets(n, k, "offgrid", seed0 + f, (8.0, 22.0), int(np.prod(b)), noise_var=nv)
        out.append(torch.from_numpy(ri.tone_cube(n, tg, nv, seed0 + f)).cuda())
    return out


def _singles(plan, cubes):
    res = []
    for x in cubes:
        loc = torch.zeros(CAP, dtype=torch.int64, device="cuda")
        amp = torch.zeros(CAP, dtype=torch.complex64, device="cuda")
        c = R.rsft_execute(plan, x, located=loc, amp=amp, allow_capacity=True)
        res.append((c, loc[:min(c, CAP)].cpu().numpy(), amp[:min(c, CAP)].cpu().numpy()))
    return res


def _frames(plan, seq, graph=False):
    n = len(seq)
    loc = torch.full((n * CAP,), -1, dtype=torch.int64, device="cuda")
    amp = torch.zeros(n * CAP, dtype=torch.complex64, device="cuda")
    counts = torch.zeros(n, dtype=torch.int64, device="cuda")
    if graph:
        g = R.rsft_graph_create_frames(plan, seq, counts, located=loc, amp=amp)
        g.launch()
        torch.cuda.synchronize()
        counts.zero_()
        loc.fill_(-1)
        g.launch()
    else:
        R.rsft_execute_frames(plan, seq, counts, located=loc, amp=amp)
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    lv, av = loc.cpu().numpy(), amp.cpu().numpy()
    return [(int(c[f]), lv[f * CAP:f * CAP + min(c[f], CAP)], av[f * CAP:f * CAP + min(c[f], CAP)]) for f in range(n)]


CASES = [
    # name, n, b, loops, extra descriptor arguments
    ("c3_small_shape", (256, 128, 16), (16, 8, 1), 10, dict(p_fa1=0.01, mu=3)),
    ("c3_mid_shape", (512, 256, 32), (32, 16, 2), 10, dict(p_fa1=0.01, mu=3)),
    ("3d_radar_small", (128, 64, 64), (16, 8, 8), 12, dict(p_fa1=0.01, mu=3)),
    ("2d_rows_of_512", (256, 512), (16, 32), 8, dict(p_fa1=0.02, mu=2)),   # wide vote rows: frames in turn
    ("3d_estimate", (128, 64, 64), (16, 8, 8), 12, dict(p_fa1=0.01, mu=3, noise_var=0.0)),
]


@pytest.mark.parametrize("name,n,b,loops,extra", CASES, ids=[c[0] for c in CASES])
def test_frames_equal_single_executes(name, n, b, loops, extra):
    plan = R.rsft_plan_create(R.make_desc(n, b, loops, seed=77, max_located=CAP, **extra))
    # every case but the wide-row one runs its frames together (small vote rows, cluster FFT, direct fold)
    assert R.rsft_plan_frames_together(plan) == (name != "2d_rows_of_512")
    cubes = _cubes(n, b, 3)
    seq = [cubes[f % 3] for f in range(19)]          # two launch groups: 16 + 3 frames
    ref = _singles(plan, cubes)
    got = _frames(plan, seq)
    for f, (c, loc, amp) in enumerate(got):
        rc, rloc, ramp = ref[f % 3]
        assert c == rc, (f, c, rc)
        np.testing.assert_array_equal(loc, rloc)
        np.testing.assert_array_equal(amp, ramp)
    assert any(r[0] > 0 for r in ref)


def test_frames_graph_and_oracle():
    n, b, loops = (256, 128, 16), (16, 8, 1), 10
    nv = 1.0
    d = R.make_desc(n, b, loops, seed=91, p_fa1=0.01, mu=3, noise_var=nv, max_located=CAP)
    plan = R.rsft_plan_create(d)
    cubes = _cubes(n, b, 2, nv=nv, seed0=500)
    seq = [cubes[0], cubes[1], cubes[0]]
    got = _frames(plan, seq, graph=True)
    ref = _singles(plan, cubes)
    for f, (c, loc, amp) in enumerate(got):
        assert c == ref[f % 2][0]
        np.testing.assert_array_equal(loc, ref[f % 2][1])
        np.testing.assert_array_equal(amp, ref[f % 2][2])
    # frame 1 against the oracle, every stage (through a single execute on the same plan geometry)
    op = O.make_plan(n, b, loops, seed=91, pfa1=0.01, mu=3, noise_var=nv)
    cube = cubes[1].cpu().numpy()
    rep = compare_full(gpu_run(d, cube), O.rsft(op, cube.astype(np.complex128)), op)
    assert rep["located"] > 0
    o = O.rsft(op, cube.astype(np.complex128))
    keep = np.isin(o["located"], got[1][1])
    assert keep.mean() > 0.99


def test_frames_one_after_another_when_not_together():
    """Scatter votes (and other plans whose stages take one frame) run the frames in turn, with
    the same results."""
    n, b, loops = (128, 64, 64), (16, 8, 8), 12
    plan = R.rsft_plan_create(R.make_desc(n, b, loops, seed=5, p_fa1=0.01, mu=3, max_located=CAP,
                                          vote_mode=R.RSFT_VOTES_SCATTER))
    assert not R.rsft_plan_frames_together(plan)
    cubes = _cubes(n, b, 2, seed0=700)
    got = _frames(plan, [cubes[1], cubes[0]])
    ref = _singles(plan, cubes)
    for f, (c, loc, amp) in enumerate(got):
        rc, rloc, ramp = ref[1 - f]
        assert c == rc
        np.testing.assert_array_equal(loc, rloc)
        np.testing.assert_array_equal(amp, ramp)


def test_frames_argument_errors():
    plan = R.rsft_plan_create(R.make_desc((64, 64), (8, 8), 4, seed=1, p_fa1=0.05, mu=1, max_located=16))
    x = torch.zeros(64 * 64 + 1, dtype=torch.complex64, device="cuda")
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    loc = torch.zeros(32, dtype=torch.int64, device="cuda")
    with pytest.raises(R.RsftError) as ei:
        R.rsft_execute_frames(plan, [x[1:].data_ptr(), x[:-1]], counts, located=loc)   # misaligned cube
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG
    with pytest.raises(R.RsftError) as ei:
        R.rsft_execute_frames(plan, [x[:-1]], counts)                                   # no located list
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG
    R.rsft_execute_frames(plan, [], counts, located=loc)                                # nothing to do
