"""Plans used from several host threads at once.  The kernels' launch attributes (dynamic
shared-memory limits, cached occupancies) are process-wide; they are set under one lock and a
limit is only ever raised, so two threads whose plans launch the same kernels with different
shared-memory sizes must each get the results a single thread gets."""
import threading

import numpy as np
import pytest
import torch

import rsft_inputs as ri
import paper_1610_01050_gb300 as R
from paper_1610_01050_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    R.load_library()


CAP = 1 << 14
# two geometries on the same fold instantiation (12 loops) with different shared-memory layouts,
# and a third with another loop count
CASES = [((128, 64, 64), (16, 8, 8), 12), ((256, 256), (16, 32), 12), ((64, 32, 16), (8, 4, 4), 10)]


def _run(plan, cube, stream):
    stream.wait_stream(torch.cuda.default_stream())   # the cube was written on the default stream
    with torch.cuda.stream(stream):                    # outputs initialised on the stream that uses them
        loc = torch.zeros(CAP, dtype=torch.int64, device="cuda")
        amp = torch.zeros(CAP, dtype=torch.complex64, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        R.rsft_execute_async(plan, cube, count, stream=stream, located=loc, amp=amp)
    stream.synchronize()
    c = int(count.item())
    return c, loc[:min(c, CAP)].cpu().numpy(), amp[:min(c, CAP)].cpu().numpy()


def test_plans_on_concurrent_threads_match_one_thread():
    plans, cubes = [], []
    for i, (n, b, loops) in enumerate(CASES):
        # each thread creates and uses its own plan; the reference runs are single-threaded first
        plans.append(R.rsft_plan_create(R.make_desc(n, b, loops, seed=10 + i, p_fa1=0.02, mu=2, max_located=CAP)))
        tg = ri.draw_targets(n, 5, "offgrid", 20 + i, (10.0, 20.0), int(np.prod(b)))
        cubes.append(torch.from_numpy(ri.tone_cube(n, tg, 1.0, 20 + i)).cuda())
    ref = [_run(p, x, torch.cuda.Stream()) for p, x in zip(plans, cubes)]
    errors, results = [], [[] for _ in CASES]

    def worker(i):
        try:
            stream = torch.cuda.Stream()
            for _ in range(25):
                results[i].append(_run(plans[i], cubes[i], stream))
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(CASES))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i, runs in enumerate(results):
        assert len(runs) == 25
        for c, loc, amp in runs:
            assert c == ref[i][0]
            np.testing.assert_array_equal(loc, ref[i][1])
            np.testing.assert_array_equal(amp, ref[i][2])


def test_new_plans_created_on_concurrent_threads():
    """Plan creation (table uploads, attribute setting on first use) from several threads at once."""
    errors, counts = [], [None] * 4

    def worker(i):
        try:
            n, b, loops = CASES[i % len(CASES)]
            plan = R.rsft_plan_create(R.make_desc(n, b, loops, seed=40 + i, p_fa1=0.02, mu=2, max_located=CAP))
            tg = ri.draw_targets(n, 4, "offgrid", 60 + i, (12.0, 20.0), int(np.prod(b)))
            x = torch.from_numpy(ri.tone_cube(n, tg, 1.0, 60 + i)).cuda()
            counts[i] = _run(plan, x, torch.cuda.Stream())[0]
            serial = _run(plan, x, torch.cuda.Stream())[0]
            assert serial == counts[i]
        except Exception as e:
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert all(c is not None and c >= 0 for c in counts)
