"""RSFT on the SRUR radar cubes of §VI (eq. (r_i); Table III system, Table IV targets): the
bursts of a Swerling-I target scene in segment mode (one burst per loop), and one burst in the
plain mode, against the oracle element by element, and the four targets located."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1610_01050_gb300 as R
import rsft_inputs as ri
from tests.gpu_helpers import compare_full, gpu_run
from tests.test_gpu_segments import _gpu_segments

pytestmark = pytest.mark.gpu

SYS = ri.SrurSystem()
B = (64, 16, 8)
BURSTS = 8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1610_01050_gb300 import build as Bld
    Bld.build()
    R.load_library()


def _hits(located, freqs):
    n = np.asarray(SYS.shape)
    idx = np.stack(np.unravel_index(located, SYS.shape), axis=1) if len(located) else np.zeros((0, 3), int)
    hits = []
    for f in freqs:
        d = np.abs(idx - np.rint(f * n).astype(int) % n)
        d = np.minimum(d, n - d)
        hits.append(bool(np.any(np.all(d <= 1, axis=1))))
    return hits


@pytest.mark.parametrize("scene", ["equal", "mixed"])
def test_srur_segment_mode(scene):
    seed = 4000 + (scene == "mixed")
    cubes, freqs, _ = ri.srur_bursts(SYS, ri.TABLE_IV[scene], BURSTS, seed=seed)
    kw = dict(atten_db=60.0, p_fa=1e-6, k_max=4, noise_var=1.0)
    desc = R.make_desc(SYS.shape, B, BURSTS, seed=seed, max_located=1 << 18, **kw)
    g = _gpu_segments(desc, cubes)
    op = O.make_plan(SYS.shape, B, BURSTS, seed=seed, **kw)
    ref = O.rsft(op, [c.astype(np.complex128) for c in cubes])
    rep = compare_full(g, ref, op)
    hits = _hits(g["located"], freqs)
    print(f"srur {scene} segments: {rep}, targets located {hits}")
    assert all(hits)


def test_srur_one_burst():
    cubes, freqs, _ = ri.srur_bursts(SYS, ri.TABLE_IV["equal"], 1, seed=4100)
    kw = dict(atten_db=60.0, p_fa=1e-6, k_max=4, noise_var=1.0)
    g = gpu_run(R.make_desc(SYS.shape, B, BURSTS, seed=4100, max_located=1 << 18, **kw), cubes[0])
    op = O.make_plan(SYS.shape, B, BURSTS, seed=4100, **kw)
    ref = O.rsft(op, cubes[0].astype(np.complex128))
    rep = compare_full(g, ref, op)
    hits = _hits(g["located"], freqs)
    print(f"srur one burst: {rep}, targets located {hits}")
    assert all(hits)
