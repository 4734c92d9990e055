"""The C ABI without a GPU: library loads, exports every declared symbol, builds
host-only plans whose tables match the oracle, and rejects bad descriptors."""
import ctypes
import re
import os

import numpy as np
import pytest

import oracle as O
import paper_1610_01050_gb300 as R
from paper_1610_01050_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return R.load_library()


def test_exports_every_declared_symbol(lib):
    header = open(os.path.join(ROOT, "include", "rsft.h")).read()
    declared = set(re.findall(r"\b(rsft_[a-z0-9_]+)\s*\(", header))
    assert declared == set(R.C_SYMBOLS)
    for name in declared:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for s in range(8):
        assert R.rsft_status_string(s) and R.rsft_status_string(s) != "unknown status"


CASES = [
    dict(n=(256, 256), b=(16, 16), loops=8, atten=60.0, flat="cheb", support=(64, 64), k=8, pfa=1e-4),
    dict(n=(1024, 256, 64), b=(64, 32, 8), loops=12, atten=80.0, flat="cheb", support=None, k=32, pfa=1e-6),
    dict(n=(64, 32, 16, 8), b=(8, 4, 2, 2), loops=16, atten=60.0, flat="ideal", support=None, k=2, pfa=1e-5),
    dict(n=(4096,), b=(64,), loops=5, atten=45.0, flat="cheb", support=(512,), k=3, pfa=1e-6),
    dict(n=(64, 64), b=(8, 8), loops=255, atten=60.0, flat="cheb", support=None, k=2, pfa=1e-6),  # largest L
]


@pytest.mark.parametrize("c", CASES, ids=[str(c["n"]) for c in CASES])
def test_host_plan_matches_oracle(lib, c):
    flat = R.RSFT_FLAT_CHEB if c["flat"] == "cheb" else R.RSFT_FLAT_IDEAL
    d = R.make_desc(c["n"], c["b"], c["loops"], atten_db=c["atten"], flat=flat, flat_support=c["support"],
                    p_fa=c["pfa"], k_max=c["k"], seed=1234, device=-1)
    p = R.rsft_plan_create(d)
    op = O.make_plan(c["n"], c["b"], c["loops"], seed=1234, atten_db=c["atten"], flat=c["flat"],
                     flat_support=c["support"], p_fa=c["pfa"], k_max=c["k"])
    np.testing.assert_array_equal(R.rsft_plan_get(p, R.RSFT_GET_SIGMA), op.sigma)
    np.testing.assert_array_equal(R.rsft_plan_get(p, R.RSFT_GET_SIGMA_INV), op.sigma_inv)
    # Chebyshev samples T_{n-1}(x0 cos(pi k / n)) near |x| = 1 have a condition number of
    # about n / sqrt(x0^2 - 1) (~3e6 at n = 4096, 45 dB): two correct FP64 routes agree to ~1e-10.
    np.testing.assert_allclose(R.rsft_plan_get(p, R.RSFT_GET_WINDOW), np.concatenate(op.w), atol=1e-9)
    fl = R.rsft_plan_get(p, R.RSFT_GET_FLAT).reshape(-1, 2)
    ofl = np.concatenate(op.wbar)
    assert np.max(np.abs(fl[:, 0] + 1j * fl[:, 1] - ofl)) < 1e-9 * np.max(np.abs(ofl))
    np.testing.assert_allclose(R.rsft_plan_get(p, R.RSFT_GET_BETA), op.beta, rtol=1e-8)
    np.testing.assert_allclose(R.rsft_plan_get(p, R.RSFT_GET_GAMMA), op.gamma, rtol=1e-8)
    assert int(R.rsft_plan_get(p, R.RSFT_GET_MU)[0]) == op.mu
    assert abs(R.rsft_plan_get(p, R.RSFT_GET_PFA1)[0] / op.pfa1 - 1) < 1e-8
    assert abs(R.rsft_plan_get(p, R.RSFT_GET_ETA_M)[0] / op.eta_m - 1) < 1e-8


BINOMIAL_CASES = [
    dict(n=(1024, 256, 64), b=(64, 32, 8), loops=12, atten=80.0, k=32, pfa=1e-6),
    dict(n=(256, 128, 16), b=(16, 8, 1), loops=10, atten=60.0, k=2, pfa=1e-5),
    dict(n=(512, 512), b=(64, 64), loops=24, atten=60.0, k=40, pfa=1e-7),
    dict(n=(64, 64), b=(8, 8), loops=255, atten=60.0, k=2, pfa=1e-6),
]


@pytest.mark.parametrize("c", BINOMIAL_CASES, ids=[str(c["n"]) + "_L" + str(c["loops"]) for c in BINOMIAL_CASES])
def test_binomial_design_matches_oracle(lib, c):
    """The binomial vote law of the threshold design: the host plan's (mu, Pfa1-bar, Pd-bar) are the
    oracle's (an independent FP64 route: scipy's binomial tail against the library's log-space sum)."""
    d = R.make_desc(c["n"], c["b"], c["loops"], atten_db=c["atten"], p_fa=c["pfa"], k_max=c["k"], seed=7,
                    device=-1, design_mode=R.RSFT_DESIGN_BINOMIAL)
    p = R.rsft_plan_create(d)
    op = O.make_plan(c["n"], c["b"], c["loops"], seed=7, atten_db=c["atten"], p_fa=c["pfa"], k_max=c["k"],
                     design_mode="binomial")
    assert int(R.rsft_plan_get(p, R.RSFT_GET_MU)[0]) == op.mu
    assert abs(R.rsft_plan_get(p, R.RSFT_GET_PFA1)[0] / op.pfa1 - 1) < 1e-8
    assert abs(R.rsft_plan_get(p, R.RSFT_GET_PD_BAR)[0] / op.design["pd_bar"] - 1) < 1e-8
    np.testing.assert_allclose(R.rsft_plan_get(p, R.RSFT_GET_GAMMA), op.gamma, rtol=1e-8)
    normal = R.rsft_plan_create(R.make_desc(c["n"], c["b"], c["loops"], atten_db=c["atten"], p_fa=c["pfa"],
                                            k_max=c["k"], seed=7, device=-1))
    assert int(R.rsft_plan_get(p, R.RSFT_GET_MU)[0]) >= int(R.rsft_plan_get(normal, R.RSFT_GET_MU)[0])


def test_estimate_mode_host_plan(lib):
    """noise_var <= 0: the plan leaves the thresholds to each execute (NaN until then)."""
    for nv in (0.0, -1.0):
        p = R.rsft_plan_create(R.make_desc((64, 128), (16, 16), 6, p_fa1=0.02, mu=2, noise_var=nv, device=-1))
        assert np.all(np.isnan(R.rsft_plan_get(p, R.RSFT_GET_GAMMA)))
        assert np.all(np.isnan(R.rsft_plan_get(p, R.RSFT_GET_GAMMA_LAST)))
        op = O.make_plan((64, 128), (16, 16), 6, pfa1=0.02, mu=2, noise_var=nv)
        assert op.estimate_noise
        np.testing.assert_allclose(R.rsft_plan_get(p, R.RSFT_GET_BETA), op.beta, rtol=1e-8)
    known = R.rsft_plan_create(R.make_desc((64, 128), (16, 16), 6, p_fa1=0.02, mu=2, noise_var=2.0, device=-1))
    np.testing.assert_array_equal(R.rsft_plan_get(known, R.RSFT_GET_GAMMA_LAST),
                                  R.rsft_plan_get(known, R.RSFT_GET_GAMMA))


def test_explicit_sigma_and_overrides(lib):
    sig = np.array([[3, 5], [7, 9], [1, 31]], dtype=np.int64)
    d = R.make_desc((32, 64), (4, 8), 3, sigma=sig, p_fa1=0.01, mu=1, noise_var=2.0, device=-1)
    p = R.rsft_plan_create(d)
    np.testing.assert_array_equal(R.rsft_plan_get(p, R.RSFT_GET_SIGMA), sig)
    inv = R.rsft_plan_get(p, R.RSFT_GET_SIGMA_INV)
    assert np.all((sig * inv) % np.array([32, 64]) == 1)
    assert int(R.rsft_plan_get(p, R.RSFT_GET_MU)[0]) == 1
    op = O.make_plan((32, 64), (4, 8), 3, sigma=sig, pfa1=0.01, mu=1, noise_var=2.0)
    np.testing.assert_allclose(R.rsft_plan_get(p, R.RSFT_GET_GAMMA), op.gamma, rtol=1e-10)


def test_design_snr_matches_oracle(lib):
    n, b = (1024,), (64,)
    d = R.make_desc(n, b, 50, atten_db=40.0, p_fa=1e-6, p_d=0.9, k_max=4, device=-1)
    p = R.rsft_plan_create(d)
    op = O.make_plan(n, b, 50, atten_db=40.0, p_fa=1e-6, p_d=0.9, k_max=4)
    ab = O.mean_alpha(op.wbar, op.w, list(b), [2 * np.pi * (1024 / 16 + 0.5) / 1024])
    bb = O.mean_beta(op.wbar, op.w)
    snr = 10 * np.log10((bb / ab) * (np.log(op.pfa1) / np.log(op.design["pd_bar"]) - 1))
    assert abs(R.rsft_plan_get(p, R.RSFT_GET_SNR_DB)[0] - snr) < 1e-8


@pytest.mark.parametrize("kw,status", [
    (dict(n=(30, 64), b=(2, 8), loops=4), R.RSFT_ERR_INVALID_ARG),        # not a power of two
    (dict(n=(32, 64), b=(64, 8), loops=4), R.RSFT_ERR_INVALID_ARG),       # B > N
    (dict(n=(32, 64), b=(4, 8), loops=0), R.RSFT_ERR_INVALID_ARG),        # no loops
    (dict(n=(32, 64), b=(4, 8), loops=256), R.RSFT_ERR_INVALID_ARG),      # votes overflow 8 bits
    (dict(n=(32, 64), b=(4, 8), loops=4, flat_support=(3, 0)), R.RSFT_ERR_INVALID_ARG),
    (dict(n=(32, 64), b=(4, 8), loops=4, mu=4, p_fa1=0.1), R.RSFT_ERR_INVALID_ARG),
    (dict(n=(32, 64), b=(4, 8), loops=4, noise_var=float("nan")), R.RSFT_ERR_INVALID_ARG),
    (dict(n=(32, 64), b=(4, 8), loops=4, noise_var=float("inf")), R.RSFT_ERR_INVALID_ARG),
    (dict(n=(32, 64), b=(4, 8), loops=4, design_mode=7), R.RSFT_ERR_INVALID_ARG),
    (dict(n=(32, 64), b=(4, 8), loops=4, sigma=[[2, 3]] * 4), R.RSFT_ERR_INVALID_ARG),  # even sigma
    (dict(n=(64, 64), b=(4, 4), loops=12, k_max=64, p_fa=1e-9), R.RSFT_ERR_DESIGN),    # K eta_m >= B
])
def test_invalid_descriptors(lib, kw, status):
    kw = dict(kw)
    d = R.make_desc(kw.pop("n"), kw.pop("b"), kw.pop("loops"), device=-1, **kw)
    with pytest.raises(R.RsftError) as ei:
        R.rsft_plan_create(d)
    assert ei.value.status == status
    assert R.rsft_last_error()


def test_ndim_limits(lib):
    d = R.rsft_desc_init()
    d.ndim = 5
    d.device = -1
    with pytest.raises(R.RsftError) as ei:
        R.rsft_plan_create(d)
    assert ei.value.status == R.RSFT_ERR_UNSUPPORTED
    d.ndim = 0
    with pytest.raises(R.RsftError) as ei:
        R.rsft_plan_create(d)
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG


def test_host_plan_cannot_execute(lib):
    p = R.rsft_plan_create(R.make_desc((32, 64), (4, 8), 3, p_fa1=0.01, mu=1, device=-1))
    cube = np.zeros((32, 64), dtype=np.complex64)
    with pytest.raises(R.RsftError) as ei:
        R.rsft_execute(p, cube.ctypes.data)   # an address: the plan refuses before any device access
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG


def test_sparsity_limit_warning(lib):
    p = R.rsft_plan_create(R.make_desc((64, 64), (4, 4), 8, k_max=64, p_fa1=0.01, mu=3, device=-1))
    assert int(R.rsft_plan_get(p, R.RSFT_GET_WARNINGS)[0]) & R.RSFT_WARN_SPARSITY_LIMIT


@pytest.mark.parametrize("field,value", [("p_fa", 0.0), ("p_fa", 1.0), ("noise_var", 0.0), ("ndim", 5)])
def test_bartlett_plan_rejects_invalid_descriptors(field, value):
    d = R.make_desc((64, 64), (8, 8), 4)
    setattr(d, field, value)
    with pytest.raises(R.RsftError) as ei:
        R.rsft_bartlett_plan_create(d)
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG


def test_bartlett_plan_rejects_non_power_of_two():
    d = R.make_desc((64, 64), (8, 8), 4)
    d.n[1] = 48
    with pytest.raises(R.RsftError) as ei:
        R.rsft_bartlett_plan_create(d)
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG


def test_batches_need_a_device_plan():
    d = R.make_desc((64, 64), (8, 8), 4, device=-1, p_fa1=0.05, mu=1)
    plan = R.rsft_plan_create(d)
    counts = np.zeros(1, dtype=np.int64)
    with pytest.raises(R.RsftError) as ei:
        R.rsft_execute_host_batch(plan, [np.zeros(64 * 64, np.complex64)], np.zeros(8, np.int64), counts)
    assert ei.value.status == R.RSFT_ERR_INVALID_ARG


def test_graphs_and_autotune_need_a_device_plan():
    """Graph recording and the fold autotuner check their arguments before touching a device."""
    plan = R.rsft_plan_create(R.make_desc((64, 64), (8, 8), 4, device=-1, p_fa1=0.05, mu=1))
    cube = np.zeros(64 * 64, np.complex64)
    count = np.zeros(1, np.int64)
    located = np.zeros(8, np.int64)
    for call in (lambda: R.rsft_graph_create(plan, cube.ctypes.data, count.ctypes.data, located.ctypes.data),
                 lambda: R.rsft_plan_autotune(plan, cube.ctypes.data)):
        with pytest.raises(R.RsftError) as ei:
            call()
        assert ei.value.status == R.RSFT_ERR_INVALID_ARG
    lib = R.load_library()
    h = ctypes.c_void_p()
    assert lib.rsft_graph_create(None, None, 0, None, None, None, ctypes.byref(h)) == R.RSFT_ERR_INVALID_ARG
    assert lib.rsft_graph_create(plan.handle, R._ptr(cube), 9, R._ptr(located), None, R._ptr(count),
                                 ctypes.byref(h)) == R.RSFT_ERR_INVALID_ARG   # lane outside 0..7
    assert lib.rsft_graph_launch(None, None) == R.RSFT_ERR_INVALID_ARG
    assert lib.rsft_graph_launch_batch(None, 0, None) == R.RSFT_OK           # empty batch: nothing to do
    assert lib.rsft_graph_launch_batch(None, -1, None) == R.RSFT_ERR_INVALID_ARG
    assert lib.rsft_plan_autotune(plan.handle, R._ptr(cube), None, 0, 10, None, None) == R.RSFT_ERR_INVALID_ARG
    lib.rsft_graph_destroy(None)  # NULL is a no-op


def test_loops_per_pass_checks_arguments():
    lib = R.load_library()
    assert lib.rsft_plan_set_loops_per_pass(None, 4) == R.RSFT_ERR_INVALID_ARG
    plan = R.rsft_plan_create(R.make_desc((64, 64), (8, 8), 4, device=-1, p_fa1=0.05, mu=1))
    assert lib.rsft_plan_set_loops_per_pass(plan.handle, 4) == R.RSFT_ERR_INVALID_ARG  # host-only plan


def test_wait_check_rejects_limits_out_of_range():
    assert R.rsft_check_wait_timeout(0) == R.RSFT_ERR_INVALID_ARG
    assert R.rsft_check_wait_timeout(1001) == R.RSFT_ERR_INVALID_ARG


class _FakeTensor:
    """Stands for a torch tensor on the given side (only the attributes the binding reads)."""

    def __init__(self, cuda):
        self.is_cuda = cuda
        self.shape = (4,)

    def data_ptr(self):
        return 1 << 40


def test_binding_refuses_memory_of_the_wrong_side():
    """Device arguments must be CUDA tensors (or raw addresses) and host arguments host memory:
    the binding raises TypeError before the library sees a pointer of the wrong kind."""
    import torch
    plan = R.rsft_plan_create(R.make_desc((64, 64), (8, 8), 4, device=-1, p_fa1=0.05, mu=1))
    host_np, host_t, dev = np.zeros(64 * 64, np.complex64), torch.zeros(64 * 64, dtype=torch.complex64), _FakeTensor(True)
    for bad in (host_np, host_t, _FakeTensor(False)):
        for call in (lambda: R.rsft_execute(plan, bad),
                     lambda: R.rsft_execute_async(plan, bad, None),
                     lambda: R.rsft_execute_segments(plan, [bad]),
                     lambda: R.rsft_execute_batch(plan, [bad], None),
                     lambda: R.rsft_copy_buckets(plan, R.RSFT_BUCKETS_FOLDED, bad),
                     lambda: R.rsft_copy_detections(plan, bad),
                     lambda: R.rsft_refine_prepare(plan, bad),
                     lambda: R.rsft_refine_eval(plan, bad, host_t[:4]),
                     lambda: R.rsft_stage2_static(bad, 16384, 1, None, None, capacity=8),
                     lambda: R.rsft_graph_create(plan, bad, None),
                     lambda: R.rsft_plan_autotune(plan, bad)):
            with pytest.raises(TypeError, match="CUDA tensor"):
                call()
    with pytest.raises(TypeError, match="host memory"):
        R.rsft_execute_host(plan, dev, np.zeros(8, np.uint64))
    with pytest.raises(TypeError, match="host memory"):
        R.rsft_execute_host_batch(plan, [host_np], dev, np.zeros(1, np.int64))
