"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Small cases run the oracle on the whole cube and compare every stage element by
element (several fold tiles, ragged chunks, both fold schedules, loop groups,
1-D to 4-D, degenerate bucket dimensions).  Full-size benchmark workloads run
in the launch configuration the benchmark times; the oracle either runs in
full or checks sampled buckets one by one, plus properties that hold at any
size.
"""
import zlib

import numpy as np
import pytest
import torch

import oracle as O
import rsft_inputs as ri
import paper_1610_01050_gb300 as R
from paper_1610_01050_gb300 import build as B
from tests.gpu_helpers import gpu_run, compare_full, rel_err, compare_tables, REL_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    R.load_library()


def make_pair(n, b, loops, *, seed, atten=60.0, window="cheb", flat="cheb", support=None, noise_var=1.0,
              pfa1=None, mu=None, p_fa=1e-6, k_max=8, max_located=65536, vote_mode=R.RSFT_VOTES_ROWS):
    d = R.make_desc(n, b, loops, window=R.RSFT_WIN_CHEB if window == "cheb" else R.RSFT_WIN_RECT,
                    atten_db=atten, flat=R.RSFT_FLAT_CHEB if flat == "cheb" else R.RSFT_FLAT_IDEAL,
                    flat_support=support, p_fa=p_fa, k_max=k_max, p_fa1=pfa1, mu=mu, noise_var=noise_var,
                    seed=seed, max_located=max_located, vote_mode=vote_mode)
    op = O.make_plan(n, b, loops, seed=seed, window=window, atten_db=atten, flat=flat, flat_support=support,
                     noise_var=noise_var, p_fa=p_fa, k_max=k_max, pfa1=pfa1, mu=mu)
    return d, op


def tone_input(n, b, k, seed, snr=(8.0, 20.0), noise_var=1.0, kind="offgrid"):
    tg = ri.draw_targets(n, k, kind, seed, snr, int(np.prod(b)), noise_var=noise_var)
    return ri.tone_cube(n, tg, noise_var, seed), tg


SMALL = [
    # name, n, b, loops, extra
    ("2d_256_cheb", (256, 256), (16, 16), 8, dict(pfa1=0.02, mu=2)),
    ("3d_rows", (64, 32, 16), (8, 4, 4), 5, dict(pfa1=0.03, mu=1)),
    ("1d", (4096,), (64,), 3, dict(pfa1=0.05, mu=1)),
    ("2d_col_chunks", (64, 2048), (8, 128), 6, dict(pfa1=0.02, mu=2)),
    ("4d_lg16", (16, 16, 8, 8), (4, 4, 2, 2), 16, dict(pfa1=0.05, mu=4)),
    ("2d_two_groups", (64, 64), (8, 8), 20, dict(pfa1=0.05, mu=5)),
    ("3d_b1", (32, 16, 16), (8, 4, 1), 6, dict(pfa1=0.05, mu=2)),
    ("2d_m1", (16, 64), (16, 4), 4, dict(pfa1=0.05, mu=1)),
    ("2d_rect_ideal", (128, 64), (16, 8), 7, dict(window="rect", flat="ideal", pfa1=0.02, mu=3)),
    ("2d_flat_support", (256, 256), (16, 16), 8, dict(support=(64, 64), pfa1=0.02, mu=2)),
    ("3d_design", (128, 64, 32), (16, 8, 4), 12, dict(atten=80.0, p_fa=1e-5, k_max=4)),
    ("4d_rows_chunked", (16, 32, 64, 32), (4, 8, 8, 4), 9, dict(pfa1=0.03, mu=2)),
    # whole 64-column rows: the tensor-core fold (rank-3 and rank-5 boxes, two loop groups)
    ("2d_tc", (512, 64), (16, 16), 4, dict(pfa1=0.02, mu=1)),
    ("3d_tc", (128, 32, 64), (16, 4, 8), 12, dict(pfa1=0.03, mu=3)),
    ("3d_tc_two_groups", (32, 64, 64), (4, 8, 4), 20, dict(pfa1=0.05, mu=5)),
]


@pytest.mark.parametrize("name,n,b,loops,extra", SMALL, ids=[c[0] for c in SMALL])
def test_parity_small(name, n, b, loops, extra):
    seed = zlib.crc32(name.encode()) % 1000
    nv = 1.5
    d, op = make_pair(n, b, loops, seed=seed, noise_var=nv, **extra)
    cube, _ = tone_input(n, b, 6, seed, noise_var=nv)
    g = gpu_run(d, cube)
    ref = O.rsft(op, cube.astype(np.complex128))
    rep = compare_full(g, ref, op)
    print(f"parity {name}: {rep}")
    assert rep["detected"] > 0


# loop counts above 32 take the shared-memory median kernel; at L = 255 the 8-bit votes reach their top
LARGE_L = [
    ("2d_l33", (64, 64), (8, 8), 33, dict(pfa1=0.05, mu=8)),
    ("3d_l64", (32, 16, 16), (8, 4, 4), 64, dict(pfa1=0.04, mu=12)),
    ("2d_l255", (64, 32), (8, 8), 255, dict(pfa1=0.05, mu=40)),
]


@pytest.mark.parametrize("name,n,b,loops,extra", LARGE_L, ids=[c[0] for c in LARGE_L])
def test_parity_large_loop_counts(name, n, b, loops, extra):
    seed = zlib.crc32(name.encode()) % 1000
    nv = 1.5
    d, op = make_pair(n, b, loops, seed=seed, noise_var=nv, **extra)
    cube, _ = tone_input(n, b, 4, seed, snr=(15.0, 25.0), noise_var=nv)
    g = gpu_run(d, cube)
    ref = O.rsft(op, cube.astype(np.complex128))
    rep = compare_full(g, ref, op)
    print(f"parity {name}: {rep}, max votes {int(ref['votes'].max())}")
    assert rep["located"] > 0


def test_votes_reach_255():
    """Noise-free on-grid tones with rectangular and ideal windows are detected in every loop: their
    votes are L = 255, the top of the 8-bit count, and their amplitudes are recovered exactly."""
    n, b, loops = (64, 64), (8, 8), 255
    tg = ri.draw_targets(n, 3, "ongrid", 17, (30.0, 30.0), int(np.prod(b)), amp_model="unit")
    cube = ri.tone_cube(n, tg, 0.0, 17)
    d, op = make_pair(n, b, loops, seed=17, window="rect", flat="ideal", pfa1=1e-3, mu=254, noise_var=1e-6)
    g = gpu_run(d, cube)
    truth = np.sort(np.ravel_multi_index(tg.grid_index(n).T, n))
    np.testing.assert_array_equal(g["located"], truth)
    assert np.all(g["located_votes"] == 255)
    assert np.all(g["votes"].reshape(-1)[truth] == 255)
    ref = O.rsft(op, cube.astype(np.complex128))
    np.testing.assert_array_equal(ref["located"], truth)
    assert rel_err(g["amp"], ref["amplitudes"]) <= REL_TOL


TC_CASES = [c for c in SMALL if c[0] in ("2d_tc", "3d_tc", "3d_tc_two_groups", "4d_lg16")]


@pytest.mark.parametrize("name,n,b,loops,extra", TC_CASES, ids=[c[0] for c in TC_CASES])
def test_tensor_core_fold_and_simt_fold(name, n, b, loops, extra, monkeypatch):
    """Both fold kernels (the default SIMT FP32 and the opt-in tcgen05 3xTF32) meet the oracle on the
    same plan geometry."""
    seed = zlib.crc32(name.encode()) % 1000 + 3
    nv = 1.5
    cube, _ = tone_input(n, b, 6, seed, noise_var=nv)
    outs = {}
    for kind in ("tc", "simt"):
        if kind == "tc":
            monkeypatch.setenv("RSFT_FOLD", "tc")
        else:
            monkeypatch.delenv("RSFT_FOLD", raising=False)
        d, op = make_pair(n, b, loops, seed=seed, noise_var=nv, **extra)
        g = gpu_run(d, cube)
        mode = int(R.rsft_plan_get(g["plan"], R.RSFT_GET_FOLD_COPY)[0])
        assert (mode >= 100) == (kind == "tc"), (kind, mode)
        outs[kind] = g
    ref = O.rsft(op, cube.astype(np.complex128))
    for kind, g in outs.items():
        rep = compare_full(g, ref, op)
        print(f"{name} {kind}: {rep}")
    assert rel_err(outs["tc"]["folded"], outs["simt"]["folded"], axis_rms=True) < 2 * REL_TOL


VOTE_CASES = [
    ("3d_rows", (64, 32, 16), (8, 4, 4), 5, dict(pfa1=0.03, mu=1)),
    ("2d_col_chunks", (64, 2048), (8, 128), 6, dict(pfa1=0.02, mu=2)),
    ("4d_lg16", (16, 16, 8, 8), (4, 4, 2, 2), 16, dict(pfa1=0.05, mu=4)),
    ("1d", (4096,), (64,), 3, dict(pfa1=0.05, mu=1)),
    ("3d_b1", (32, 16, 16), (8, 4, 1), 6, dict(pfa1=0.05, mu=2)),
]


@pytest.mark.parametrize("name,n,b,loops,extra", VOTE_CASES, ids=[c[0] for c in VOTE_CASES])
def test_vote_modes_agree_with_oracle(name, n, b, loops, extra):
    """Row-organised votes and the atomic scatter give the oracle's votes and located set."""
    seed = zlib.crc32(name.encode()) % 1000 + 7
    nv = 1.5
    cube, _ = tone_input(n, b, 6, seed, noise_var=nv)
    outs = []
    for mode in (R.RSFT_VOTES_ROWS, R.RSFT_VOTES_SCATTER):
        d, op = make_pair(n, b, loops, seed=seed, noise_var=nv, vote_mode=mode, **extra)
        g = gpu_run(d, cube)
        outs.append(g)
    ref = O.rsft(op, cube.astype(np.complex128))
    for g in outs:
        compare_full(g, ref, op)
    np.testing.assert_array_equal(outs[0]["votes"], outs[1]["votes"])
    np.testing.assert_array_equal(outs[0]["located"], outs[1]["located"])


def test_parity_config1_workload():
    """The 2-D 256 x 256 workload in full: 8 on-grid tones, flat support 4 N / B = 64."""
    cube, tg, wl, nv = ri.workload_frame("c1_2d_256")
    d, op = make_pair(wl.shape, wl.buckets, wl.loops, seed=101, atten=wl.atten_db, support=wl.flat_support,
                      noise_var=nv, p_fa=wl.p_fa, k_max=8)
    g = gpu_run(d, cube)
    ref = O.rsft(op, cube.astype(np.complex128))
    rep = compare_full(g, ref, op)
    assert rep["located"] > 0


def test_empty_and_zero_inputs():
    n, b = (64, 128), (8, 16)
    d, op = make_pair(n, b, 6, seed=3, pfa1=1e-300, mu=5)
    cube = ri.tone_cube(n, None, 1.0, 9)
    g = gpu_run(d, cube)
    assert g["count"] == 0 and not g["detected"].any() and not g["votes"].any()
    d2, _ = make_pair(n, b, 6, seed=3, pfa1=0.5, mu=0)
    g2 = gpu_run(d2, np.zeros(n, dtype=np.complex64))
    assert g2["count"] == 0 and not g2["detected"].any()
    assert np.all(g2["folded"] == 0)


def test_capacity_overflow_keeps_ascending_prefix():
    n, b = (128, 128), (8, 8)
    d, op = make_pair(n, b, 6, seed=5, pfa1=0.2, mu=0, max_located=7)
    cube, _ = tone_input(n, b, 5, 5)
    plan = R.rsft_plan_create(d)
    x = torch.from_numpy(cube).cuda()
    loc = torch.zeros(7, dtype=torch.int64, device="cuda")
    with pytest.raises(R.RsftError) as ei:
        R.rsft_execute(plan, x, located=loc)
    assert ei.value.status == R.RSFT_ERR_CAPACITY
    cnt = R.rsft_execute(plan, x, located=loc, allow_capacity=True)
    ref = O.rsft(op, cube.astype(np.complex128), estimate=False)
    assert cnt == len(ref["located"]) > 7
    np.testing.assert_array_equal(loc.cpu().numpy(), ref["located"][:7])


def test_repeat_calls_identical_and_votes_cleared():
    n, b = (128, 64, 16), (16, 8, 4)
    d, op = make_pair(n, b, 10, seed=8, pfa1=0.05, mu=3)
    cube, _ = tone_input(n, b, 8, 8)
    plan = R.rsft_plan_create(d)
    x = torch.from_numpy(cube).cuda()
    outs = []
    for _ in range(3):
        loc = torch.zeros(65536, dtype=torch.int64, device="cuda")
        amp = torch.zeros(65536, dtype=torch.complex64, device="cuda")
        votes = torch.zeros(int(np.prod(n)), dtype=torch.uint8, device="cuda")
        c = R.rsft_execute(plan, x, located=loc, amp=amp, votes_out=votes)
        outs.append((c, loc[:c].cpu().numpy(), amp[:c].cpu().numpy(), votes.cpu().numpy()))
    for o in outs[1:]:
        assert o[0] == outs[0][0]
        np.testing.assert_array_equal(o[1], outs[0][1])
        np.testing.assert_array_equal(o[2], outs[0][2])   # deterministic reduction order
        np.testing.assert_array_equal(o[3], outs[0][3])


def test_misaligned_cube_rejected():
    n, b = (64, 64), (8, 8)
    d, _ = make_pair(n, b, 4, seed=1, pfa1=0.1, mu=1)
    plan = R.rsft_plan_create(d)
    buf = torch.zeros(64 * 64 + 1, dtype=torch.complex64, device="cuda")
    loc = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(R.RsftError) as ei:
        R.rsft_execute(plan, buf[1:].data_ptr(), located=loc)
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG


def test_async_and_host_entry_points_agree():
    n, b = (128, 128), (16, 16)
    d, op = make_pair(n, b, 8, seed=21, pfa1=0.03, mu=2)
    cube, _ = tone_input(n, b, 6, 21)
    plan = R.rsft_plan_create(d)
    x = torch.from_numpy(cube).cuda()
    loc = torch.zeros(65536, dtype=torch.int64, device="cuda")
    amp = torch.zeros(65536, dtype=torch.complex64, device="cuda")
    cnt_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    R.rsft_execute_async(plan, x, cnt_dev, located=loc, amp=amp)
    torch.cuda.synchronize()
    c = int(cnt_dev.item())
    h_loc = np.zeros(65536, dtype=np.uint64)
    h_amp = np.zeros(65536, dtype=np.complex64)
    c2 = R.rsft_execute_host(plan, cube, h_loc, h_amp)
    assert c == c2
    np.testing.assert_array_equal(loc[:c].cpu().numpy().astype(np.uint64), h_loc[:c])
    np.testing.assert_array_equal(amp[:c].cpu().numpy(), h_amp[:c])
    ref = O.rsft(op, cube.astype(np.complex128))
    np.testing.assert_array_equal(h_loc[:c].astype(np.int64), ref["located"])


# ---------------------------------------------------------------- full-size workloads

def _full_oracle_case(name, frame=0):
    cube, tg, wl, nv = ri.workload_frame(name, frame)
    d, op = make_pair(wl.shape, wl.buckets, wl.loops, seed=ri.frame_seed(wl, frame), atten=wl.atten_db,
                      support=wl.flat_support, noise_var=nv, p_fa=wl.p_fa,
                      k_max=wl.k_design, max_located=1 << 20)
    g = gpu_run(d, cube)
    ref = O.rsft(op, cube.astype(np.complex128))
    return compare_full(g, ref, op), g, ref, tg, wl


@pytest.mark.parametrize("name", ["c2_3d_radar", "c3_small", "c3_mid", "c3_large", "c4_2d_4096"])
def test_parity_full_workload(name):
    rep, g, ref, tg, wl = _full_oracle_case(name)
    print(f"parity {name}: {rep}")
    assert rep["detected"] > 0 and rep["located"] > 0


def test_parity_full_workload_binomial_design():
    """The radar workload under the binomial vote-law design (the bench's matched operating point)."""
    cube, tg, wl, nv = ri.workload_frame("c2_3d_radar")
    seed = ri.frame_seed(wl, 0)
    d = R.make_desc(wl.shape, wl.buckets, wl.loops, seed=seed, atten_db=wl.atten_db, noise_var=nv, p_fa=wl.p_fa,
                    k_max=wl.k_design, max_located=1 << 20, design_mode=R.RSFT_DESIGN_BINOMIAL)
    op = O.make_plan(wl.shape, wl.buckets, wl.loops, seed=seed, atten_db=wl.atten_db, noise_var=nv, p_fa=wl.p_fa,
                     k_max=wl.k_design, design_mode="binomial")
    g = gpu_run(d, cube)
    ref = O.rsft(op, cube.astype(np.complex128))
    rep = compare_full(g, ref, op)
    print(f"parity c2_3d_radar binomial design (mu {op.mu}): {rep}")
    assert rep["located"] > 0


def test_tensor_core_fold_full_workload(monkeypatch):
    """The opt-in tcgen05 fold on the full 1024x256x64 radar workload, every stage against the oracle."""
    monkeypatch.setenv("RSFT_FOLD", "tc")
    rep, g, ref, tg, wl = _full_oracle_case("c2_3d_radar")
    assert int(R.rsft_plan_get(g["plan"], R.RSFT_GET_FOLD_COPY)[0]) >= 100
    print(f"parity c2_3d_radar (tensor-core fold): {rep}")
    assert rep["detected"] > 0 and rep["located"] > 0


def test_parity_c5_sampled():
    """4-D 512 x 512 x 64 x 32 (4.3 GB): sampled buckets against eq. (l) one by one; sampled
    spectrum values, detections, votes and amplitudes against the oracle's bucket spectrum at the
    sampled (loop, bucket) pairs (oracle.spectrum_at: eq. (l) and the bucket DFT as one sum over the
    cube); plus properties over the whole output (Parseval per loop, votes from the detections by
    Def. 3, located = votes > mu)."""
    name = "c5_4d"
    cube, tg, wl, nv = ri.workload_frame(name, 0)
    d, op = make_pair(wl.shape, wl.buckets, wl.loops, seed=ri.frame_seed(wl, 0), atten=wl.atten_db,
                      noise_var=nv, p_fa=wl.p_fa, k_max=wl.k_design, max_located=1 << 22)
    g = gpu_run(d, cube, want_votes=True)
    compare_tables(g["plan"], op)
    rng = np.random.default_rng(5)
    L = wl.loops
    for l in range(L):
        js = [tuple(int(rng.integers(0, bb)) for bb in wl.buckets) for _ in range(12)]
        ref = np.array([O.fold_bucket_direct(op, cube, l, j) for j in js])
        got = np.array([g["folded"][(l,) + j] for j in js])
        rms = np.sqrt(np.mean(np.abs(g["folded"][l]) ** 2))
        assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 0.1 * rms)) <= REL_TOL
    bt = int(np.prod(wl.buckets))
    for l in range(L):
        f, fh = g["folded"][l].astype(np.complex128), g["spectrum"][l].astype(np.complex128)
        assert abs(np.sum(np.abs(fh) ** 2) / (bt * np.sum(np.abs(f) ** 2)) - 1) < 1e-5     # Parseval
    votes = g["votes"]
    mtot = int(np.prod(op.m))
    assert int(votes.astype(np.int64).sum()) == int(g["detected"].sum()) * mtot
    np.testing.assert_array_equal(g["located"], np.flatnonzero(votes.reshape(-1) > op.mu))

    # the oracle's spectrum at sampled pairs: the buckets of 8 located cells (for their amplitudes and
    # votes) and of 8 random cells (votes), in every loop, plus 64 random buckets
    located = g["located"]
    pick_loc = located[rng.choice(len(located), size=min(8, len(located)), replace=False)]
    pick_rnd = rng.integers(0, np.prod(wl.shape), size=8)
    cells = [np.unravel_index(int(i), wl.shape) for i in np.concatenate([pick_loc, pick_rnd])]
    pairs = sorted({(l, O.mapping(op, l, i)) for i in cells for l in range(L)} |
                   {(int(rng.integers(0, L)), tuple(int(rng.integers(0, bb)) for bb in wl.buckets))
                    for _ in range(64)})
    vals = O.spectrum_at(op, cube, pairs)
    spec = {pk: v for pk, v in zip(pairs, vals)}
    for l in range(L):
        rms = np.sqrt(np.mean(np.abs(g["spectrum"][l]) ** 2))
        for (ll, k), v in spec.items():
            if ll != l:
                continue
            assert abs(g["spectrum"][(l,) + k] - v) <= REL_TOL * max(abs(v), 0.1 * rms), (l, k)
            p = abs(v) ** 2
            if abs(p - op.gamma[l]) > 1e-5 * op.gamma[l]:
                assert bool(g["detected"][(l,) + k]) == (p > op.gamma[l]), (l, k)
    band_cells = 0
    for i in cells:
        ps = [abs(spec[(l, O.mapping(op, l, i))]) ** 2 for l in range(L)]
        if any(abs(p - op.gamma[l]) <= 1e-5 * op.gamma[l] for l, p in enumerate(ps)):
            band_cells += 1
            continue
        assert int(votes[i]) == sum(int(p > op.gamma[l]) for l, p in enumerate(ps)), i

    class _Sampled:                       # spectra[l][k] for the sampled pairs only
        def __getitem__(self, l):
            return {k: v for (ll, k), v in spec.items() if ll == l}

    amp_ref = O.estimate_amplitudes(op, _Sampled(), pick_loc)
    pos = np.searchsorted(located, pick_loc)
    amp_gpu = g["amp"][pos]
    arms = np.sqrt(np.mean(np.abs(g["amp"]) ** 2))
    assert np.max(np.abs(amp_gpu - amp_ref) / np.maximum(np.abs(amp_ref), 0.1 * arms)) <= REL_TOL
    print(f"c5: {len(located)} located, {len(pairs)} oracle pairs, {band_cells} sampled cells in the band")
