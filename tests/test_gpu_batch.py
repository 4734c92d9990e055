"""Batched executes (several lanes, device or host buffers) give, frame for frame, exactly
the results of single executes: same kernels and arithmetic, only scheduled concurrently."""
import numpy as np
import pytest
import torch

import paper_1610_01050_gb300 as R
import rsft_inputs as ri

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1610_01050_gb300 import build as B
    B.build()
    R.load_library()


N, BK, L, CAP = (128, 64, 16), (16, 8, 4), 10, 1 << 16


def _frames(k):
    out = []
    for f in range(k):
        tg = ri.draw_targets(N, 6, "offgrid", 300 + f, (10.0, 20.0), int(np.prod(BK)))
        out.append(ri.tone_cube(N, tg, 1.0, 300 + f))
    return out


def _single(plan, cube):
    x = torch.from_numpy(cube).cuda()
    loc = torch.zeros(CAP, dtype=torch.int64, device="cuda")
    amp = torch.zeros(CAP, dtype=torch.complex64, device="cuda")
    c = R.rsft_execute(plan, x, located=loc, amp=amp)
    return c, loc[:c].cpu().numpy(), amp[:c].cpu().numpy()


@pytest.mark.parametrize("lanes", [1, 2, 3])
def test_device_batch_matches_single_executes(lanes):
    plan = R.rsft_plan_create(R.make_desc(N, BK, L, seed=5, p_fa1=0.03, mu=3, max_located=CAP))
    frames = _frames(5)
    ref = [_single(plan, f) for f in frames]
    cubes = [torch.from_numpy(f).cuda() for f in frames]
    counts = torch.full((len(frames),), -1, dtype=torch.int64, device="cuda")
    located = torch.zeros(len(frames) * CAP, dtype=torch.int64, device="cuda")
    amp = torch.zeros(len(frames) * CAP, dtype=torch.complex64, device="cuda")
    for _ in range(2):  # the second batch reuses the lanes' workspaces
        R.rsft_execute_batch(plan, cubes, counts, lanes=lanes, located=located, amp=amp)
        torch.cuda.synchronize()
        for f, (c, loc, a) in enumerate(ref):
            assert int(counts[f]) == c > 0
            np.testing.assert_array_equal(located[f * CAP:f * CAP + c].cpu().numpy(), loc)
            np.testing.assert_array_equal(amp[f * CAP:f * CAP + c].cpu().numpy(), a)


def test_host_batch_matches_single_executes():
    plan = R.rsft_plan_create(R.make_desc(N, BK, L, seed=6, p_fa1=0.03, mu=3, max_located=CAP))
    frames = _frames(4)
    ref = [_single(plan, f) for f in frames]
    hosts = [torch.from_numpy(f).pin_memory() for f in frames]
    counts = np.full(len(frames), -1, dtype=np.int64)
    located = np.zeros(len(frames) * CAP, dtype=np.int64)
    amp = np.zeros(len(frames) * CAP, dtype=np.complex64)
    R.rsft_execute_host_batch(plan, hosts, located, counts, amp=amp)
    for f, (c, loc, a) in enumerate(ref):
        assert counts[f] == c
        np.testing.assert_array_equal(located[f * CAP:f * CAP + c], loc)
        np.testing.assert_array_equal(amp[f * CAP:f * CAP + c], a)


def test_batch_rejects_bad_arguments():
    plan = R.rsft_plan_create(R.make_desc(N, BK, L, seed=5, p_fa1=0.03, mu=3, max_located=CAP))
    x = torch.zeros(int(np.prod(N)), dtype=torch.complex64, device="cuda")
    counts = torch.zeros(1, dtype=torch.int64, device="cuda")
    located = torch.zeros(CAP, dtype=torch.int64, device="cuda")
    for lanes in (0, 9):
        with pytest.raises(R.RsftError) as ei:
            R.rsft_execute_batch(plan, [x], counts, lanes=lanes, located=located)
        assert ei.value.status == R.RSFT_ERR_INVALID_ARG
    raw = torch.zeros(x.numel() * 2 + 2, dtype=torch.float32, device="cuda")
    with pytest.raises(R.RsftError) as ei:
        R.rsft_execute_batch(plan, [raw[1:]], counts, lanes=1, located=located)
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG
