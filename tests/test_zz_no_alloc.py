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

    # capacity 0 and no output list: the full count is still written and the votes cleared
    v = votes.clone()
    count.zero_()
    R.rsft_stage2_static(v, total, 3, None, count, capacity=0)
    torch.cuda.synchronize()
    assert int(count.item()) == cnt
    assert int(v.count_nonzero().item()) == 0

    # the binding refuses tensors shorter than n or the capacity before anything is launched
    v = votes.clone()
    with pytest.raises(ValueError):
        R.rsft_stage2_static(v, total + 16384, 3, loc, count)
    short_votes = torch.zeros(cap - 1 if cap > 1 else 0, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        R.rsft_stage2_static(v, total, 3, loc, count, located_votes=short_votes)
    with pytest.raises(ValueError):
        R.rsft_stage2_static(v, total, 3, loc, count, capacity=cap + 1)
    with pytest.raises(TypeError):
        R.rsft_stage2_static(v.view(torch.int8), total, 3, loc, count)
    with pytest.raises(TypeError):
        R.rsft_stage2_static(v, total, 3, loc.view(torch.float64), count)
    torch.testing.assert_close(v, votes, rtol=0, atol=0)     # nothing ran

    # the C entry point's own limits, called directly (each is rejected on the host, before a launch)
    lib = R.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    for bad_n, bad_mu in ((total + 16, 3), ((1 << 28) + (1 << 14), 3), (total, 255), (0, 3)):
        st = lib.rsft_stage2_static(v.data_ptr(), bad_n, bad_mu, loc.data_ptr(), None, cap, count.data_ptr(), stream)
        assert st == R.RSFT_ERR_INVALID_ARG, (bad_n, bad_mu, st)
    st = lib.rsft_stage2_static(v.data_ptr() + 1, total, 3, loc.data_ptr(), None, cap, count.data_ptr(), stream)
    assert st == R.RSFT_ERR_INVALID_ARG                       # misaligned votes
    st = lib.rsft_stage2_static(v.data_ptr(), total, 3, None, None, cap, count.data_ptr(), stream)
    assert st == R.RSFT_ERR_INVALID_ARG                       # a capacity without a list
    torch.testing.assert_close(v, votes, rtol=0, atol=0)
