"""Segment mode on the GPU (loop l folds its own data segment) against the oracle's segment
mode, element by element: folded buckets, spectrum, detections, votes, located list,
amplitudes (tolerances as in the single-cube parity tests)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1610_01050_gb300 as R
import rsft_inputs as ri
from tests.gpu_helpers import compare_full

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1610_01050_gb300 import build as B
    B.build()
    R.load_library()


def _gpu_segments(desc, segs):
    plan = R.rsft_plan_create(desc)
    n = tuple(int(desc.n[i]) for i in range(desc.ndim))
    b = tuple(int(desc.b[i]) for i in range(desc.ndim))
    L, cap, total_b = int(desc.loops), int(desc.max_located), int(np.prod(b))
    dsegs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in segs]
    located = torch.zeros(cap, dtype=torch.int64, device="cuda")
    lvotes = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    amp = torch.zeros(cap, dtype=torch.complex64, device="cuda")
    votes = torch.zeros(int(np.prod(n)), dtype=torch.uint8, device="cuda")
    cnt = R.rsft_execute_segments(plan, dsegs, located=located, located_votes=lvotes, amp=amp, votes_out=votes,
                                  allow_capacity=True)
    folded = torch.empty(L * total_b, dtype=torch.complex64, device="cuda")
    spectrum = torch.empty(L * total_b, dtype=torch.complex64, device="cuda")
    words = (total_b + 31) // 32
    det = torch.zeros(L * words, dtype=torch.int32, device="cuda")
    R.rsft_copy_buckets(plan, R.RSFT_BUCKETS_FOLDED, folded)
    R.rsft_copy_buckets(plan, R.RSFT_BUCKETS_SPECTRUM, spectrum)
    R.rsft_copy_detections(plan, det)
    torch.cuda.synchronize()
    k = min(cnt, cap)
    bits = np.unpackbits(det.cpu().numpy().view(np.uint8), bitorder="little").reshape(L, words * 32)[:, :total_b]
    return {"plan": plan, "count": cnt, "located": located[:k].cpu().numpy().astype(np.int64),
            "located_votes": lvotes[:k].cpu().numpy(), "amp": amp[:k].cpu().numpy(),
            "votes": votes.cpu().numpy().reshape(n), "folded": folded.cpu().numpy().reshape((L,) + b),
            "spectrum": spectrum.cpu().numpy().reshape((L,) + b), "detected": bits.reshape((L,) + b).astype(bool)}


CASES = [
    ("2d", (256, 256), (16, 16), 8, dict(pfa1=0.02, mu=2)),
    ("3d", (64, 32, 16), (8, 4, 4), 5, dict(pfa1=0.03, mu=1)),
    ("3d_l20", (64, 64, 16), (8, 8, 4), 20, dict(pfa1=0.05, mu=4)),
    ("4d", (16, 16, 8, 8), (4, 4, 2, 2), 6, dict(pfa1=0.05, mu=2)),
    ("2d_cols", (64, 2048), (8, 128), 6, dict(pfa1=0.02, mu=2)),
]


@pytest.mark.parametrize("name,n,b,loops,kw", CASES, ids=[c[0] for c in CASES])
def test_segment_mode_parity(name, n, b, loops, kw):
    seed = 500 + loops
    tg = ri.draw_targets(n, 5, "offgrid", seed, (15.0, 25.0), int(np.prod(b)))
    segs = ri.segment_cubes(n, tg, 1.0, seed, loops, int(np.prod(b)))
    desc = R.make_desc(n, b, loops, seed=seed, max_located=1 << 18, p_fa1=kw["pfa1"], mu=kw["mu"])
    g = _gpu_segments(desc, segs)
    op = O.make_plan(n, b, loops, seed=seed, pfa1=kw["pfa1"], mu=kw["mu"])
    ref = O.rsft(op, [s.astype(np.complex128) for s in segs])
    rep = compare_full(g, ref, op)
    assert rep["located"] == g["count"] or rep["band"] > 0


def test_segment_mode_mid_cube():
    # the middle batched shape, 512 x 256 x 32 with B = N / 16, ten segments
    wl = ri.WORKLOADS["c3_mid"]
    tg = ri.draw_targets(wl.shape, 16, "offgrid", 77, (5.0, 25.0), int(np.prod(wl.buckets)))
    segs = ri.segment_cubes(wl.shape, tg, 1.0, 77, wl.loops, int(np.prod(wl.buckets)))
    desc = R.make_desc(wl.shape, wl.buckets, wl.loops, seed=77, atten_db=wl.atten_db, p_fa=wl.p_fa, k_max=16,
                       max_located=1 << 20)
    g = _gpu_segments(desc, segs)
    op = O.make_plan(wl.shape, wl.buckets, wl.loops, seed=77, atten_db=wl.atten_db, p_fa=wl.p_fa, k_max=16)
    ref = O.rsft(op, [s.astype(np.complex128) for s in segs])
    compare_full(g, ref, op)


def test_segments_need_one_aligned_cube_per_loop():
    n, b, loops = (64, 64), (8, 8), 4
    plan = R.rsft_plan_create(R.make_desc(n, b, loops, seed=1, p_fa1=0.05, mu=1))
    good = torch.zeros(64 * 64, dtype=torch.complex64, device="cuda")
    raw = torch.zeros(64 * 64 * 2 + 2, dtype=torch.float32, device="cuda")
    loc = torch.zeros(65536, dtype=torch.int64, device="cuda")
    with pytest.raises(R.RsftError) as ei:
        R.rsft_execute_segments(plan, [good, good, raw[1:], good], located=loc)
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG
