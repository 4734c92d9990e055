"""The bounded device waits: every barrier wait of the kernels gives up after a time limit,
sets an error flag and lets its kernel return.  A CTA waiting on a barrier that nothing
completes (through the fold's own wait routine, limit 20 ms) must give up, the call must
report RSFT_ERR_TIMEOUT, and the context must still run an RSFT against the oracle."""
import time

import numpy as np
import pytest
import torch

import oracle as O
import paper_1610_01050_gb300 as R
import rsft_inputs as ri

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1610_01050_gb300 import build as B
    B.build()
    R.load_library()


def test_wait_gives_up_and_the_context_stays_usable():
    t0 = time.perf_counter()
    assert R.rsft_check_wait_timeout(20) == R.RSFT_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    n, b, loops = (64, 64), (8, 8), 4
    tg = ri.draw_targets(n, 3, "offgrid", 3, (15.0, 25.0), 64)
    cube = ri.tone_cube(n, tg, 1.0, 3)
    plan = R.rsft_plan_create(R.make_desc(n, b, loops, seed=3, p_fa1=0.05, mu=1))
    loc = torch.zeros(4096, dtype=torch.int64, device="cuda")
    c = R.rsft_execute(plan, torch.from_numpy(cube).cuda(), located=loc)
    ref = O.rsft(O.make_plan(n, b, loops, seed=3, pfa1=0.05, mu=1), cube.astype(np.complex128))
    np.testing.assert_array_equal(loc[:c].cpu().numpy(), ref["located"])
