"""The fold's host-side schedule (paper_1610_01050_gb300/csrc/fold_schedule.h): the work
split the plan chooses, the column pair each thread holds, the lane bits the warp shuffle
sums and the epilogue's slot lists.  The header is compiled on its own with the host C++
compiler; every property is then re-derived here by brute force over the 256 threads:
placement a bijection that keeps quarter warps on 8 consecutive pairs, shuffled lanes sharing
(class, inner residue), every partial sum listed exactly once under its own key."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1610_01050_gb300", "csrc")

# (n, b, loops): the small parity geometries, the benchmark workloads and the radar scene
GEOMETRIES = [
    ((256, 256), (16, 16), 8), ((64, 32, 16), (8, 4, 4), 5), ((4096,), (64,), 3), ((64, 2048), (8, 128), 6),
    ((16, 16, 8, 8), (4, 4, 2, 2), 16), ((64, 64), (8, 8), 20), ((32, 16, 16), (8, 4, 1), 6), ((16, 64), (16, 4), 4),
    ((128, 64), (16, 8), 7), ((128, 64, 32), (16, 8, 4), 12), ((16, 32, 64, 32), (4, 8, 8, 4), 9),
    ((512, 64), (16, 16), 4), ((128, 32, 64), (16, 4, 8), 12), ((32, 64, 64), (4, 8, 4), 20),
    ((1024, 256, 64), (64, 32, 8), 12), ((256, 128, 16), (16, 8, 1), 10), ((512, 256, 32), (32, 16, 2), 10),
    ((1024, 256, 64), (64, 16, 4), 10), ((4096, 4096), (128, 128), 16), ((512, 512, 64, 32), (32, 32, 8, 4), 16),
    ((2048, 64, 32), (64, 16, 8), 8),
]


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    if not cxx or not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("probe") / "fold_schedule_probe")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", inc,
                    os.path.join(ROOT, "tests", "host", "fold_schedule_probe.cpp"), "-o", exe], check=True)
    text = "".join(f"{len(n)} {loops} 152 {' '.join(map(str, n))} {' '.join(map(str, b))}\n" for n, b, loops in GEOMETRIES)
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.splitlines()
    assert len(out) == len(GEOMETRIES)
    res = []
    for line in out:
        assert line != "none"
        kv = dict(item.split("=", 1) for item in line.split())
        rec = {k: (v if k == "error" else [int(t) for t in v.split(",")] if k in ("slots", "digits") else int(v))
               for k, v in kv.items()}
        res.append(rec)
    return res


def _residue(n, b, d_in, col):
    """Inner residue of chunk column col (last dimension fastest)."""
    x, stride = 0, 1
    for d in range(len(n) - 1, d_in - 1, -1):
        sd = col % n[d]
        col //= n[d]
        x += (sd % b[d]) * stride
        stride *= b[d]
    return x


def _pair(t, perm):
    return sum(((t >> q) & 1) << ((perm >> (4 * q)) & 15) for q in range(8))


@pytest.mark.parametrize("i", range(len(GEOMETRIES)), ids=["x".join(map(str, g[0])) for g in GEOMETRIES])
def test_schedule_and_epilogue_tables(probe, i):
    n, b, loops = GEOMETRIES[i]
    s = probe[i]
    assert s["error"] == "no"
    d_in, w, cps, X = s["d_in"], s["width"], s["cps"], s["xcount"]
    assert X == int(np.prod(b[d_in:])) and w * s["col_chunks"] == int(np.prod(n[d_in:]))
    perm = s["lane_perm"]
    pairs = [_pair(t, perm) for t in range(256)]
    assert sorted(pairs) == list(range(256))                          # a bijection of the 256 threads
    assert all(pairs[t] & 7 == t & 7 for t in range(256))             # quarter warps: 8 consecutive pairs
    pair_bits = (w // 2).bit_length() - 1
    assert all((pairs[t] >> pair_bits) == (t >> pair_bits) for t in range(256))   # rows stay with their threads

    def key(t, c):
        e = 2 * pairs[t] + c
        return ((e // w) % cps, _residue(n, b, d_in, e % w))

    keeping = [all(key(t, c) == key(t ^ (1 << k), c) for t in range(256) for c in (0, 1)) for k in range(5)]
    rmask = s["red_mask"]
    assert rmask == sum(1 << k for k in range(5) if keeping[k])       # exactly the lane bits that keep the key
    assert s["leaders"] == 32 >> bin(rmask).count("1")
    if pair_bits > 5:                                                 # wide rows: lane bits 3-4 on kept columns
        kept_cols = sum(all(key(t, c) == key(t ^ (1 << q), c) for t in range(256) for c in (0, 1))
                        for q in range(3, pair_bits) if (perm >> (4 * q) & 15) >= 3)
        assert all(keeping[k] for k in (3, 4)[:min(2, kept_cols)])
    # slot lists: every leader's partial sum once, under its own key
    per = s["slots_per_x"]
    slots = s["slots"]
    assert len(slots) == 8 * s["leaders"] * 2 == per * cps * X
    assert sorted(slots) == list(range(len(slots)))
    free = [k for k in range(5) if not (rmask >> k) & 1]
    for kx in range(cps * X):
        for sl in slots[kx * per:(kx + 1) * per]:
            c, lead = sl % 2, sl // 2
            wv, j = divmod(lead, s["leaders"])
            lane = sum(((j >> q) & 1) << free[q] for q in range(len(free)))
            cls, x = key(32 * wv + lane, c)
            assert cls * X + x == kx
    # residue digits: mixed radix of the column dimensions, last fastest
    dig = np.asarray(s["digits"]).reshape(X, 4)
    for x in range(X):
        rem = x
        for d in range(len(n) - 1, d_in - 1, -1):
            assert dig[x, d - d_in] == rem % b[d]
            rem //= b[d]
