"""rsft_stage2_static: the second-stage detection for callers that cannot allocate.

Such callers (a real-time loop whose device memory is fixed at start-up, a host
framework that owns every allocation, code that must not trigger the device
synchronisation cudaMalloc/cudaFree may cause) hand in the vote array and the
output buffers; the entry point's only scratch is a fixed array inside the
library.  Its result must equal the located list rsft_execute produces from the
same votes, call after call, since every call reuses that one array.
"""
import numpy as np
import pytest
import torch

import paper_1610_01050_gb300 as R
from paper_1610_01050_gb300 import build as B
import rsft_inputs as ri

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    R.load_library()


def _reference_run(n, b, loops, seed):
    d = R.make_desc(n, b, loops, seed=seed, p_fa1=0.05, mu=3, max_located=1 << 18)
    plan = R.rsft_plan_create(d)
    tg = ri.draw_targets(n, 8, "offgrid", seed, (8.0, 20.0), int(np.prod(b)))
    cube = torch.from_numpy(ri.tone_cube(n, tg, 1.0, seed)).cuda()
    total = int(np.prod(n))
    located = torch.zeros(1 << 18, dtype=torch.int64, device="cuda")
    lvotes = torch.zeros(1 << 18, dtype=torch.uint8, device="cuda")
    votes = torch.zeros(total, dtype=torch.uint8, device="cuda")
    cnt = R.rsft_execute(plan, cube, located=located, located_votes=lvotes, votes_out=votes)
    return plan, votes, located[:cnt].clone(), lvotes[:cnt].clone(), cnt


def test_static_stage2_matches_execute_twice():
    n, b, loops = (128, 64, 16), (16, 8, 4), 10
    plan, votes, ref_loc, ref_lv, cnt = _reference_run(n, b, loops, 41)
    assert cnt > 0
    total = int(np.prod(n))
    for _ in range(2):                       # the shared scratch keeps the last call's contents
        v = votes.clone()
        loc = torch.full((1 << 18,), -1, dtype=torch.int64, device="cuda")
        lv = torch.zeros(1 << 18, dtype=torch.uint8, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        R.rsft_stage2_static(v, total, 3, loc, count, located_votes=lv)
        torch.cuda.synchronize()
        c = int(count.item())
        assert c == cnt
        torch.testing.assert_close(loc[:c], ref_loc, rtol=0, atol=0)
        torch.testing.assert_close(lv[:c], ref_lv, rtol=0, atol=0)
        assert int(v.count_nonzero().item()) == 0        # votes cleared, as rsft_execute does


def test_static_stage2_capacity_and_limits():
    n, b, loops = (64, 64, 16), (8, 8, 4), 8
    plan, votes, ref_loc, _, cnt = _reference_run(n, b, loops, 43)
    total = int(np.prod(n))
    cap = max(1, cnt // 2)
    loc = torch.zeros(cap, dtype=torch.int64, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    v = votes.clone()
    R.rsft_stage2_static(v, total, 3, loc, count)
    torch.cuda.synchronize()
    assert int(count.item()) == cnt
    torch.testing.assert_close(loc, ref_loc[:cap], rtol=0, atol=0)
    for bad_n in (total + 16, (1 << 28) + (1 << 14)):
        with pytest.raises(R.RsftError) as ei:
            R.rsft_stage2_static(v, bad_n, 3, loc, count)
        assert ei.value.status == R.RSFT_ERR_INVALID_ARG
    with pytest.raises(R.RsftError) as ei:
        R.rsft_stage2_static(v, total, 255, loc, count)
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG
