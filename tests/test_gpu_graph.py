"""CUDA-graph executes and the fold autotuner.  A recorded execute runs the same kernels on
the same arithmetic, so its results equal rsft_execute's bit for bit (on any lane, launch
after launch); a batch of graphs of plans of different shapes gives each frame exactly its
single-execute result; an autotuned plan (another fold schedule: only the FP32 summation
order changes) still meets the FP64 oracle at every stage."""
import zlib

import numpy as np
import pytest
import torch

import oracle as O
import paper_1610_01050_gb300 as R
import rsft_inputs as ri
from tests.gpu_helpers import gpu_run, compare_full
from tests.test_gpu_parity import make_pair

pytestmark = pytest.mark.gpu

CAP = 1 << 16
SHAPES = [((128, 64, 16), (16, 8, 4), 10), ((64, 32, 64), (8, 4, 8), 8)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1610_01050_gb300 import build as B
    B.build()
    R.load_library()


def _plan(n, b, loops, seed):
    return R.rsft_plan_create(R.make_desc(n, b, loops, p_fa=1e-5, k_max=6, seed=seed, max_located=CAP))


def _cube(n, b, seed):
    tg = ri.draw_targets(n, 6, "offgrid", seed, (10.0, 20.0), int(np.prod(b)))
    return torch.from_numpy(ri.tone_cube(n, tg, 1.0, seed)).cuda()


def _outputs():
    return (torch.zeros(CAP, dtype=torch.int64, device="cuda"), torch.zeros(CAP, dtype=torch.complex64, device="cuda"),
            torch.zeros(1, dtype=torch.int64, device="cuda"))


def _single(plan, x):
    loc, amp, _ = _outputs()
    c = R.rsft_execute(plan, x, located=loc, amp=amp)
    return c, loc[:c].cpu().numpy(), amp[:c].cpu().numpy()


@pytest.mark.parametrize("lane", [0, 3])
def test_graph_equals_execute(lane):
    n, b, loops = SHAPES[0]
    plan = _plan(n, b, loops, 11)
    x = _cube(n, b, 11)
    c, loc_ref, amp_ref = _single(plan, x)
    assert c > 0
    loc, amp, cnt = _outputs()
    g = R.rsft_graph_create(plan, x, cnt, located=loc, amp=amp, lane=lane)
    for _ in range(3):  # every launch rewrites the same outputs
        loc.zero_()
        amp.zero_()
        g.launch()
        torch.cuda.synchronize()
        k = int(cnt.item())
        assert k == c
        np.testing.assert_array_equal(loc[:k].cpu().numpy(), loc_ref)
        np.testing.assert_array_equal(amp[:k].cpu().numpy(), amp_ref)
    g.close()


def test_graph_batch_of_mixed_shapes():
    plans = [_plan(n, b, loops, 20 + i) for i, (n, b, loops) in enumerate(SHAPES)]
    frames, graphs, outs, refs = [], [], [], []
    for f in range(6):
        i = f % 2
        n, b, _ = SHAPES[i]
        x = _cube(n, b, 40 + f)
        refs.append(_single(plans[i], x))
        o = _outputs()
        graphs.append(R.rsft_graph_create(plans[i], x, o[2], located=o[0], amp=o[1], lane=(f // 2) % 3))
        frames.append(x)
        outs.append(o)
    order = [0, 1, 2, 3, 4, 5, 1, 0, 5]  # repeats run after their earlier launch on the same lane
    R.rsft_graph_launch_batch([graphs[f] for f in order])
    torch.cuda.synchronize()
    for f in range(6):
        c, loc_ref, amp_ref = refs[f]
        loc, amp, cnt = outs[f]
        assert int(cnt.item()) == c
        np.testing.assert_array_equal(loc[:c].cpu().numpy(), loc_ref)
        np.testing.assert_array_equal(amp[:c].cpu().numpy(), amp_ref)
    for g in graphs:
        g.close()


@pytest.mark.parametrize("n,b,loops", [((128, 64, 32), (16, 8, 4), 12), ((256, 128, 16), (16, 8, 1), 10)])
def test_autotuned_plan_meets_oracle(n, b, loops):
    seed = zlib.crc32(str(n).encode()) % 1000
    d, op = make_pair(n, b, loops, seed=seed, p_fa=1e-5, k_max=4, noise_var=1.5, max_located=CAP)
    tg = ri.draw_targets(n, 6, "offgrid", seed, (10.0, 20.0), int(np.prod(b)), noise_var=1.5)
    cube = ri.tone_cube(n, tg, 1.5, seed)
    plan = R.rsft_plan_create(d)
    x = torch.from_numpy(cube).cuda()
    us, chosen = R.rsft_plan_autotune(plan, x, candidates=4, reps=3)
    assert us > 0 and 0 <= chosen < 4
    g = gpu_run(d, cube_dev=x, plan=plan)
    rep = compare_full(g, O.rsft(op, cube.astype(np.complex128)), op)
    print(f"autotuned {n}: {us:.1f} us per fold, candidate {chosen}, {rep}")
    assert rep["located"] > 0


def test_graph_in_scatter_vote_mode():
    """The atomic-scatter vote path (vote array cleared inside the recorded execute) replays exactly."""
    n, b, loops = SHAPES[1]
    plan = R.rsft_plan_create(R.make_desc(n, b, loops, p_fa=1e-5, k_max=6, seed=5, max_located=CAP,
                                          vote_mode=R.RSFT_VOTES_SCATTER))
    x = _cube(n, b, 5)
    c, loc_ref, amp_ref = _single(plan, x)
    loc, amp, cnt = _outputs()
    g = R.rsft_graph_create(plan, x, cnt, located=loc, amp=amp, lane=1)
    for _ in range(2):
        g.launch()
        torch.cuda.synchronize()
        assert int(cnt.item()) == c
        np.testing.assert_array_equal(loc[:c].cpu().numpy(), loc_ref)
        np.testing.assert_array_equal(amp[:c].cpu().numpy(), amp_ref)
    g.close()


def test_autotune_then_segments_and_multipass_epilogue():
    """After autotuning, segment mode rebuilds its one-loop tables from the new schedule; a
    geometry whose fold epilogue runs in passes (512-column chunks, 64 residues, 16 loops)
    tunes and still meets the oracle."""
    n, b, loops = (256, 2048), (8, 64), 16
    seed = 77
    d, op = make_pair(n, b, loops, seed=seed, p_fa=1e-5, k_max=4, noise_var=1.5, max_located=CAP)
    tg = ri.draw_targets(n, 6, "offgrid", seed, (10.0, 20.0), int(np.prod(b)), noise_var=1.5)
    cube = ri.tone_cube(n, tg, 1.5, seed)
    plan = R.rsft_plan_create(d)
    x = torch.from_numpy(cube).cuda()
    us, chosen = R.rsft_plan_autotune(plan, x, candidates=3, reps=2)
    assert us > 0
    g = gpu_run(d, cube_dev=x, plan=plan)
    compare_full(g, O.rsft(op, cube.astype(np.complex128)), op)
    # segment mode on the tuned plan: every loop folds the same cube -> the plain result
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    loc, amp, _ = _outputs()
    R.rsft_execute_segments_async(plan, [x] * loops, count, located=loc, amp=amp)
    torch.cuda.synchronize()
    c = int(count.item())
    assert c == g["count"]
    np.testing.assert_array_equal(loc[:c].cpu().numpy().astype(np.int64), g["located"])


@pytest.mark.parametrize("lpp", [1, 4, 5])
def test_loops_per_pass_meet_oracle(lpp):
    """Folding the loops in passes of 1, 4 or 5 (the last pass ragged) gives the oracle's
    results at every stage, like the default single pass."""
    n, b, loops = (128, 64, 32), (16, 8, 4), 12
    seed = 31 + lpp
    d, op = make_pair(n, b, loops, seed=seed, p_fa=1e-5, k_max=4, noise_var=1.5, max_located=CAP)
    tg = ri.draw_targets(n, 6, "offgrid", seed, (10.0, 20.0), int(np.prod(b)), noise_var=1.5)
    cube = ri.tone_cube(n, tg, 1.5, seed)
    plan = R.rsft_plan_create(d)
    R.rsft_plan_set_loops_per_pass(plan, lpp)
    fold_bytes = int(R.rsft_plan_get(plan, R.RSFT_GET_FOLD_BYTES)[0])
    assert fold_bytes == -(-loops // lpp) * int(np.prod(n)) * 8 + loops * int(np.prod(b)) * 8
    x = torch.from_numpy(cube).cuda()
    g = gpu_run(d, cube_dev=x, plan=plan)
    rep = compare_full(g, O.rsft(op, cube.astype(np.complex128)), op)
    assert rep["located"] > 0


FFT_SHAPES = [((1024, 256, 64), (64, 32, 8), 12), ((256, 512), (128, 128), 8), ((512, 256, 32), (32, 16, 2), 10)]


@pytest.mark.parametrize("n,b,loops", FFT_SHAPES, ids=["radar", "2d_b16384", "3d_b1024"])
def test_every_fft_cluster_shape_gives_the_same_spectrum(n, b, loops):
    """The bucket FFT's cluster shape (CTAs per loop, threads per CTA) changes no arithmetic: every
    valid shape gives the default shape's spectrum, detections and located list bit for bit; an
    invalid shape is refused; the autotuner's choice is one of them."""
    d = R.make_desc(n, b, loops, seed=33, p_fa1=0.01, mu=3, max_located=1 << 18)
    tg = ri.draw_targets(n, 6, "offgrid", 33, (10.0, 20.0), int(np.prod(b)))
    cube = ri.tone_cube(n, tg, 1.0, 33)
    plan = R.rsft_plan_create(d)
    ref = gpu_run(d, cube, plan=plan, want_votes=False)
    tried = 0
    for c in (1, 2, 4, 8):
        for t in (256, 512):
            try:
                R.rsft_plan_set_fft_shape(plan, c, t)
            except R.RsftError as e:
                assert e.status == R.RSFT_ERR_UNSUPPORTED
                continue
            assert list(R.rsft_plan_get(plan, R.RSFT_GET_FFT_SHAPE)) == [c, t]
            g = gpu_run(d, cube, plan=plan, want_votes=False)
            np.testing.assert_array_equal(g["spectrum"], ref["spectrum"])
            np.testing.assert_array_equal(g["detected"], ref["detected"])
            np.testing.assert_array_equal(g["located"], ref["located"])
            tried += 1
    assert tried >= 2
    with pytest.raises(R.RsftError):
        R.rsft_plan_set_fft_shape(plan, 3, 256)
    R.rsft_plan_set_fft_shape(plan, 0, 0)
    x = torch.from_numpy(cube).cuda()
    R.rsft_plan_autotune(plan, x, candidates=2, reps=3)
    c, t = R.rsft_plan_get(plan, R.RSFT_GET_FFT_SHAPE)
    assert c in (1, 2, 4, 8) and t in (256, 512)
    g = gpu_run(d, cube, plan=plan, want_votes=False)
    np.testing.assert_array_equal(g["located"], ref["located"])
