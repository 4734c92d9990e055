"""Host-side helpers of bench.py: the detection-quality score of a located list and the
lookup of committed ncu traffic (used only when the profiled kernel source is unchanged)."""
import hashlib
import os
import types

import numpy as np
import pytest

import bench


def _targets(bins, shape):
    return types.SimpleNamespace(freqs=np.asarray(bins, dtype=np.float64) / np.asarray(shape))


def test_detection_quality_hits_wrap_around_and_false_alarms():
    shape = (64, 64)
    tg = _targets([[10, 10], [40, 63]], shape)
    located = np.ravel_multi_index(np.array([[11, 9], [40, 0], [30, 30], [12, 12]]).T, shape)
    pd, pfa = bench.detection_quality(None, tg, shape, located)
    assert pd == 1.0                                    # (11, 9) and (40, 0) across the wrap
    assert pfa == pytest.approx(1.0 / (64 * 64 - 2 * 49))   # (30, 30) only: (12, 12) is inside a +-3 box
    pd, pfa = bench.detection_quality(None, tg, shape, np.zeros(0, dtype=np.int64))
    assert (pd, pfa) == (0.0, 0.0)
    pd, _ = bench.detection_quality(None, tg, shape, np.ravel_multi_index(np.array([[13, 10]]).T, shape))
    assert pd == 0.0                                    # two bins off is not a hit


def test_profile_traffic_needs_the_profiled_source(tmp_path, monkeypatch):
    src = tmp_path / "paper_1610_01050_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "fold.cu").write_text("// kernel v1\n")
    (tmp_path / "profiles").mkdir()
    digest = hashlib.sha256(b"// kernel v1\n").hexdigest()[:16]
    (tmp_path / "profiles" / "permute_window_fold_wl.txt").write_text(
        f"title line\nsource: fold.cu\nsource_sha256_16: {digest}\ndram_bytes_per_launch: 1234\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("wl", "fold.cu") == 1234.0
    (src / "fold.cu").write_text("// kernel v2\n")
    assert bench.profile_traffic("wl", "fold.cu") is None        # counters of another build
    assert bench.profile_traffic("other", "fold.cu") is None     # no summary for this workload
