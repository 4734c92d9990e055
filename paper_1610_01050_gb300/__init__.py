"""GB300-native RSFT hot path: a thin Python binding of the C ABI in include/rsft.h.

The functions here have the names of the C entry points and only marshal
arguments (torch tensors or numpy arrays to pointers and sizes); every step of
the path runs in the CUDA library ``_lib/librsft.so``.  There is no CPU
fallback: if the library is missing, or no GPU is present, calls raise.

Typical use::

    import torch, paper_1610_01050_gb300 as R
    desc = R.make_desc(n=(1024, 256, 64), b=(64, 32, 8), loops=12, atten_db=80.0, p_fa=1e-6, k_max=32)
    plan = R.rsft_plan_create(desc)
    cube = torch.randn(1024, 256, 64, dtype=torch.complex64, device="cuda")
    located = torch.empty(desc.max_located, dtype=torch.int64, device="cuda")
    amp = torch.empty(desc.max_located, dtype=torch.complex64, device="cuda")
    n = R.rsft_execute(plan, cube, located=located, amp=amp)
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_size_t, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librsft.so")

RSFT_OK, RSFT_ERR_INVALID_ARG, RSFT_ERR_UNSUPPORTED, RSFT_ERR_OOM = 0, 1, 2, 3
RSFT_ERR_CAPACITY, RSFT_ERR_CUDA, RSFT_ERR_TIMEOUT, RSFT_ERR_DESIGN = 4, 5, 6, 7
RSFT_WIN_RECT, RSFT_WIN_CHEB = 0, 1
RSFT_FLAT_IDEAL, RSFT_FLAT_CHEB = 0, 1
RSFT_BETA_EXACT, RSFT_BETA_MEAN = 0, 1
RSFT_VOTES_ROWS, RSFT_VOTES_SCATTER = 0, 1
RSFT_DESIGN_NORMAL, RSFT_DESIGN_BINOMIAL = 0, 1
RSFT_WARN_SPARSITY_LIMIT = 1
RSFT_GET_SIGMA, RSFT_GET_SIGMA_INV, RSFT_GET_GAMMA, RSFT_GET_BETA = 1, 2, 3, 4
RSFT_GET_MU, RSFT_GET_PFA1, RSFT_GET_ETA_M, RSFT_GET_PD_BAR = 5, 6, 7, 8
RSFT_GET_WINDOW, RSFT_GET_FLAT, RSFT_GET_WARNINGS, RSFT_GET_SNR_DB = 9, 10, 11, 12
RSFT_GET_WORKSPACE_BYTES, RSFT_GET_STAGE_MS, RSFT_GET_FOLD_BYTES, RSFT_GET_FOLD_COPY = 13, 14, 15, 16
RSFT_GET_GAMMA_LAST, RSFT_GET_FRAMES_FOLD, RSFT_GET_FFT_SHAPE = 17, 18, 19
RSFT_BUCKETS_FOLDED, RSFT_BUCKETS_SPECTRUM = 0, 1

# Every C entry point declared in include/rsft.h.
C_SYMBOLS = (
    "rsft_desc_init", "rsft_plan_create", "rsft_plan_destroy", "rsft_execute",
    "rsft_execute_async", "rsft_execute_host", "rsft_plan_get", "rsft_plan_timing", "rsft_copy_buckets",
    "rsft_copy_detections", "rsft_refine", "rsft_refine_prepare", "rsft_refine_eval", "rsft_stage2_static", "rsft_status_string",
    "rsft_last_error", "rsft_execute_batch", "rsft_execute_host_batch", "rsft_execute_segments",
    "rsft_execute_segments_async", "rsft_bartlett_plan_create", "rsft_bartlett_plan_destroy", "rsft_bartlett_execute",
    "rsft_bartlett_execute_async", "rsft_bartlett_get", "rsft_bartlett_copy_spectrum",
    "rsft_graph_create", "rsft_graph_launch", "rsft_graph_launch_batch", "rsft_graph_destroy", "rsft_plan_autotune",
    "rsft_plan_set_loops_per_pass", "rsft_check_wait_timeout", "rsft_execute_frames", "rsft_plan_frames_together",
    "rsft_graph_create_frames", "rsft_plan_set_fft_shape",
)
RSFT_BARTLETT_GAMMA, RSFT_BARTLETT_GAIN, RSFT_BARTLETT_WINDOW, RSFT_BARTLETT_WORKSPACE_BYTES = 1, 2, 3, 4


class RsftDesc(ctypes.Structure):
    """Mirror of ``struct rsft_desc``."""
    _fields_ = [
        ("ndim", c_int32), ("n", c_int64 * 4), ("b", c_int64 * 4), ("loops", c_int32),
        ("window", c_int32), ("atten_db", c_double), ("flat", c_int32),
        ("flat_support", c_int64 * 4), ("p_fa", c_double), ("p_d", c_double),
        ("k_max", c_int32), ("eta_p", c_double), ("p_fa1_override", c_double),
        ("mu_override", c_int32), ("noise_var", c_double), ("seed", c_uint64),
        ("sigma", POINTER(c_int64)), ("beta_mode", c_int32), ("max_located", c_int64),
        ("device", c_int32), ("vote_mode", c_int32), ("design_mode", c_int32),
    ]


class RsftError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librsft.so (built by ``paper_1610_01050_gb300.build.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1610_01050_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    lib.rsft_desc_init.argtypes = [POINTER(RsftDesc)]
    lib.rsft_desc_init.restype = None
    lib.rsft_plan_create.argtypes = [POINTER(RsftDesc), POINTER(c_void_p)]
    lib.rsft_plan_destroy.argtypes = [c_void_p]
    lib.rsft_plan_destroy.restype = None
    lib.rsft_execute.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 POINTER(c_int64)]
    lib.rsft_execute_async.argtypes = [c_void_p] * 8
    lib.rsft_execute_host.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int64)]
    lib.rsft_plan_get.argtypes = [c_void_p, c_int32, c_void_p, c_size_t]
    lib.rsft_plan_timing.argtypes = [c_void_p, c_int32]
    lib.rsft_copy_buckets.argtypes = [c_void_p, c_int32, c_void_p, c_void_p]
    lib.rsft_copy_detections.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.rsft_refine.argtypes = [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_int32, ctypes.c_float,
                                c_void_p]
    lib.rsft_refine_prepare.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.rsft_refine_eval.argtypes = [c_void_p, c_int64] + [c_void_p] * 7
    lib.rsft_stage2_static.argtypes = [c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_int64, c_void_p,
                                       c_void_p]
    lib.rsft_execute_segments.argtypes = [c_void_p, POINTER(c_void_p), c_void_p, c_void_p, c_void_p, c_void_p,
                                          c_void_p, POINTER(c_int64)]
    lib.rsft_execute_segments_async.argtypes = [c_void_p, POINTER(c_void_p)] + [c_void_p] * 6
    lib.rsft_execute_batch.argtypes = [c_void_p, POINTER(c_void_p), c_int64, c_int32, c_void_p, c_void_p, c_void_p,
                                       c_void_p]
    lib.rsft_execute_host_batch.argtypes = [c_void_p, POINTER(c_void_p), c_int64, c_void_p, c_void_p, c_void_p,
                                            c_void_p]
    lib.rsft_bartlett_plan_create.argtypes = [POINTER(RsftDesc), POINTER(c_void_p)]
    lib.rsft_bartlett_plan_destroy.argtypes = [c_void_p]
    lib.rsft_bartlett_plan_destroy.restype = None
    lib.rsft_bartlett_execute.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int64)]
    lib.rsft_bartlett_execute_async.argtypes = [c_void_p] * 6
    lib.rsft_bartlett_get.argtypes = [c_void_p, c_int32, c_void_p, c_size_t]
    lib.rsft_bartlett_copy_spectrum.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.rsft_graph_create.argtypes = [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p, POINTER(c_void_p)]
    lib.rsft_graph_launch.argtypes = [c_void_p, c_void_p]
    lib.rsft_execute_frames.argtypes = [c_void_p, POINTER(c_void_p), c_int64, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.rsft_plan_frames_together.argtypes = [c_void_p, POINTER(c_int32)]
    lib.rsft_plan_set_fft_shape.argtypes = [c_void_p, c_int32, c_int32]
    lib.rsft_graph_create_frames.argtypes = [c_void_p, POINTER(c_void_p), c_int64, c_void_p, c_void_p, c_void_p,
                                             POINTER(c_void_p)]
    lib.rsft_graph_launch_batch.argtypes = [POINTER(c_void_p), c_int64, c_void_p]
    lib.rsft_graph_destroy.argtypes = [c_void_p]
    lib.rsft_graph_destroy.restype = None
    lib.rsft_plan_autotune.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_int32, POINTER(ctypes.c_double),
                                       POINTER(c_int32)]
    lib.rsft_plan_set_loops_per_pass.argtypes = [c_void_p, c_int32]
    lib.rsft_check_wait_timeout.argtypes = [c_int32, c_void_p]
    lib.rsft_check_wait_timeout.restype = c_int32
    lib.rsft_status_string.argtypes = [c_int32]
    lib.rsft_status_string.restype = c_char_p
    lib.rsft_last_error.argtypes = []
    lib.rsft_last_error.restype = c_char_p
    for name in ("rsft_plan_create", "rsft_execute", "rsft_execute_async", "rsft_execute_host",
                 "rsft_plan_get", "rsft_plan_timing", "rsft_copy_buckets", "rsft_copy_detections",
                 "rsft_refine", "rsft_stage2_static", "rsft_execute_frames", "rsft_plan_frames_together",
                 "rsft_graph_create_frames", "rsft_plan_set_fft_shape"):
        getattr(lib, name).restype = c_int32
    _lib = lib
    return lib


def _check(status: int, allow=()):
    if status != RSFT_OK and status not in allow:
        lib = load_library()
        raise RsftError(status, f"{lib.rsft_status_string(status).decode()}: {lib.rsft_last_error().decode()}")
    return status


def _ptr(x):
    """Device or host pointer of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return c_void_p(x.ctypes.data)
    if isinstance(x, int):
        return c_void_p(x)
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _dptr(x, what):
    """Device pointer of a CUDA tensor (None -> NULL; an int is taken as a device address).
    Host memory is refused here: the kernels would read it as device memory."""
    if x is None:
        return None
    if isinstance(x, int):
        return c_void_p(x)
    if hasattr(x, "is_cuda") and x.is_cuda:
        return c_void_p(x.data_ptr())
    kind = "a CPU tensor" if hasattr(x, "is_cuda") else type(x).__name__
    raise TypeError(f"{what} must be a CUDA tensor (device memory), not {kind}")


def _hptr(x, what):
    """Host pointer of a numpy array or CPU tensor (None -> NULL; an int is taken as a host address)."""
    if x is None:
        return None
    if isinstance(x, int):
        return c_void_p(x)
    if isinstance(x, np.ndarray):
        return c_void_p(x.ctypes.data)
    if hasattr(x, "is_cuda") and not x.is_cuda:
        return c_void_p(x.data_ptr())
    kind = "a CUDA tensor" if hasattr(x, "is_cuda") else type(x).__name__
    raise TypeError(f"{what} must be host memory (a numpy array or CPU tensor), not {kind}")


def _dptr_array(xs, what):
    return (c_void_p * max(1, len(xs)))(*[_dptr(x, what).value for x in xs])


def _hptr_array(xs, what):
    return (c_void_p * max(1, len(xs)))(*[_hptr(x, what).value for x in xs])


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return c_void_p(stream.cuda_stream)
    return c_void_p(int(stream))


class Plan:
    """Owning handle of an ``rsft_plan``; keeps the descriptor (and sigma table) alive."""

    def __init__(self, handle: c_void_p, desc: RsftDesc, keep=None):
        self.handle = handle
        self.desc = desc
        self._keep = keep

    @property
    def shape(self):
        return tuple(int(self.desc.n[i]) for i in range(self.desc.ndim))

    @property
    def buckets(self):
        return tuple(int(self.desc.b[i]) for i in range(self.desc.ndim))

    @property
    def loops(self):
        return int(self.desc.loops)

    def close(self):
        if self.handle:
            load_library().rsft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rsft_desc_init() -> RsftDesc:
    d = RsftDesc()
    load_library().rsft_desc_init(ctypes.byref(d))
    return d


def make_desc(n, b, loops, *, window=RSFT_WIN_CHEB, atten_db=60.0, flat=RSFT_FLAT_CHEB, flat_support=None,
              p_fa=1e-6, p_d=0.9, k_max=8, eta_p=1.0, p_fa1=None, mu=None, noise_var=1.0, seed=0,
              sigma=None, beta_mode=RSFT_BETA_EXACT, max_located=65536, device=0,
              vote_mode=RSFT_VOTES_ROWS, design_mode=RSFT_DESIGN_NORMAL) -> RsftDesc:
    """Descriptor from keyword arguments (sizes per dimension, powers of two).  ``noise_var <= 0``
    selects the estimate mode of the first stage (noise floor from each loop's bucket powers)."""
    d = rsft_desc_init()
    d.ndim = len(n)
    for i, (nn, bb) in enumerate(zip(n, b)):
        d.n[i] = int(nn)
        d.b[i] = int(bb)
    d.loops = int(loops)
    d.window = int(window)
    d.atten_db = float(atten_db)
    d.flat = int(flat)
    if flat_support is not None:
        for i, s in enumerate(flat_support):
            d.flat_support[i] = int(s)
    d.p_fa, d.p_d, d.k_max, d.eta_p = float(p_fa), float(p_d), int(k_max), float(eta_p)
    d.p_fa1_override = float(p_fa1) if p_fa1 is not None else -1.0
    d.mu_override = int(mu) if mu is not None else -1
    d.noise_var = float(noise_var)
    d.seed = int(seed) & ((1 << 64) - 1)
    d.beta_mode = int(beta_mode)
    d.max_located = int(max_located)
    d.device = int(device)
    d.vote_mode = int(vote_mode)
    d.design_mode = int(design_mode)
    if sigma is not None:
        arr = np.ascontiguousarray(np.asarray(sigma, dtype=np.int64).reshape(-1))
        d._sigma_keep = arr
        d.sigma = arr.ctypes.data_as(POINTER(c_int64))
    return d


def rsft_plan_create(desc: RsftDesc) -> Plan:
    lib = load_library()
    h = c_void_p()
    _check(lib.rsft_plan_create(ctypes.byref(desc), ctypes.byref(h)))
    return Plan(h, desc, keep=getattr(desc, "_sigma_keep", None))


def rsft_plan_destroy(plan: Plan) -> None:
    plan.close()


def rsft_execute(plan: Plan, cube, stream=None, located=None, located_votes=None, amp=None,
                 votes_out=None, allow_capacity=False) -> int:
    """Run the hot path on a device cube; returns the number of located frequencies."""
    n = c_int64(0)
    st = load_library().rsft_execute(plan.handle, _dptr(cube, "cube"), _stream(stream), _dptr(located, "located"),
                                     _dptr(located_votes, "located_votes"), _dptr(amp, "amp"),
                                     _dptr(votes_out, "votes_out"), ctypes.byref(n))
    _check(st, allow=(RSFT_ERR_CAPACITY,) if allow_capacity else ())
    return int(n.value)


def rsft_execute_async(plan: Plan, cube, count, stream=None, located=None, located_votes=None, amp=None,
                       votes_out=None) -> None:
    """Stream-ordered run; the located count lands in the device int64 tensor ``count``."""
    _check(load_library().rsft_execute_async(plan.handle, _dptr(cube, "cube"), _stream(stream),
                                             _dptr(located, "located"), _dptr(located_votes, "located_votes"),
                                             _dptr(amp, "amp"), _dptr(votes_out, "votes_out"),
                                             _dptr(count, "count")))


def rsft_execute_host(plan: Plan, h_cube, located, amp=None, stream=None, allow_capacity=False) -> int:
    """End-to-end run on host buffers (numpy or CPU torch; pinned memory recommended)."""
    n = c_int64(0)
    st = load_library().rsft_execute_host(plan.handle, _hptr(h_cube, "h_cube"), _stream(stream),
                                          _hptr(located, "located"), _hptr(amp, "amp"),
                                          ctypes.byref(n))
    _check(st, allow=(RSFT_ERR_CAPACITY,) if allow_capacity else ())
    return int(n.value)


_GET_SHAPES = {
    RSFT_GET_SIGMA: ("int64", "ld"), RSFT_GET_SIGMA_INV: ("int64", "ld"),
    RSFT_GET_GAMMA: ("float64", "l"), RSFT_GET_BETA: ("float64", "l"),
    RSFT_GET_MU: ("int32", "1"), RSFT_GET_PFA1: ("float64", "1"), RSFT_GET_ETA_M: ("float64", "1"),
    RSFT_GET_PD_BAR: ("float64", "1"), RSFT_GET_WINDOW: ("float64", "sn"),
    RSFT_GET_FLAT: ("float64", "2sn"), RSFT_GET_WARNINGS: ("int32", "1"),
    RSFT_GET_SNR_DB: ("float64", "1"), RSFT_GET_WORKSPACE_BYTES: ("int64", "1"),
    RSFT_GET_STAGE_MS: ("float64", "8"), RSFT_GET_FOLD_BYTES: ("int64", "1"), RSFT_GET_FOLD_COPY: ("int32", "1"),
    RSFT_GET_GAMMA_LAST: ("float64", "l"), RSFT_GET_FRAMES_FOLD: ("float64", "3"), RSFT_GET_FFT_SHAPE: ("int32", "2"),
}


def _ptr_array(xs):
    return (c_void_p * max(1, len(xs)))(*[_ptr(x).value for x in xs])


def rsft_execute_segments(plan: Plan, segments, stream=None, located=None, located_votes=None, amp=None,
                          votes_out=None, allow_capacity=False) -> int:
    """Segment mode: loop l folds segments[l] (one device cube per loop); returns the count."""
    n = c_int64(0)
    st = load_library().rsft_execute_segments(plan.handle, _dptr_array(segments, "segments"), _stream(stream),
                                              _dptr(located, "located"), _dptr(located_votes, "located_votes"),
                                              _dptr(amp, "amp"), _dptr(votes_out, "votes_out"), ctypes.byref(n))
    _check(st, allow=(RSFT_ERR_CAPACITY,) if allow_capacity else ())
    return int(n.value)


def rsft_execute_segments_async(plan: Plan, segments, count, stream=None, located=None, located_votes=None,
                                amp=None, votes_out=None) -> None:
    _check(load_library().rsft_execute_segments_async(plan.handle, _dptr_array(segments, "segments"),
                                                      _stream(stream), _dptr(located, "located"),
                                                      _dptr(located_votes, "located_votes"), _dptr(amp, "amp"),
                                                      _dptr(votes_out, "votes_out"), _dptr(count, "count")))


def rsft_execute_batch(plan: Plan, cubes, counts, lanes: int = 2, located=None, amp=None, stream=None) -> None:
    """Stream-ordered batch of device cubes over `lanes` lanes; frame f's count lands in
    counts[f], its located list in located[f * max_located:], its amplitudes likewise."""
    _check(load_library().rsft_execute_batch(plan.handle, _dptr_array(cubes, "cubes"), len(cubes), lanes,
                                             _stream(stream), _dptr(located, "located"), _dptr(amp, "amp"),
                                             _dptr(counts, "counts")))


def rsft_execute_frames(plan: Plan, cubes, counts, located=None, amp=None, stream=None) -> None:
    """Frames of the plan's shape in one launch per stage (16 frames per launch); frame f's
    count lands in counts[f], its located list in located[f * max_located:], its amplitudes
    likewise.  Stream-ordered."""
    _check(load_library().rsft_execute_frames(plan.handle, _dptr_array(cubes, "cubes"), len(cubes), _stream(stream),
                                              _dptr(located, "located"), _dptr(amp, "amp"), _dptr(counts, "counts")))


def rsft_plan_set_fft_shape(plan: Plan, ctas_per_loop: int, threads: int) -> None:
    """Bucket FFT cluster shape (CTAs per loop 1/2/4/8, threads 256/512); 0, 0 restores the default."""
    _check(load_library().rsft_plan_set_fft_shape(plan.handle, int(ctas_per_loop), int(threads)))


def rsft_plan_frames_together(plan: Plan) -> bool:
    """Whether rsft_execute_frames runs this plan's frames together (else one after another)."""
    out = c_int32(0)
    _check(load_library().rsft_plan_frames_together(plan.handle, ctypes.byref(out)))
    return bool(out.value)


def rsft_execute_host_batch(plan: Plan, h_cubes, located, counts, amp=None, stream=None, allow_capacity=False) -> None:
    """Host cubes in, host results out (counts[f], located[f * max_located:], amp likewise)."""
    st = load_library().rsft_execute_host_batch(plan.handle, _hptr_array(h_cubes, "h_cubes"), len(h_cubes),
                                                _stream(stream), _hptr(located, "located"), _hptr(amp, "amp"),
                                                _hptr(counts, "counts"))
    _check(st, allow=(RSFT_ERR_CAPACITY,) if allow_capacity else ())


def rsft_plan_get(plan: Plan, what: int) -> np.ndarray:
    dt, kind = _GET_SHAPES[what]
    d = plan.desc
    L, D = int(d.loops), int(d.ndim)
    sn = sum(int(d.n[i]) for i in range(D))
    count = {"ld": L * D, "l": L, "1": 1, "2": 2, "3": 3, "8": 8, "sn": sn, "2sn": 2 * sn}[kind]
    out = np.zeros(count, dtype=dt)
    _check(load_library().rsft_plan_get(plan.handle, int(what), _ptr(out), out.nbytes))
    if kind == "ld":
        return out.reshape(L, D)
    return out


def rsft_plan_timing(plan: Plan, enable: bool) -> None:
    _check(load_library().rsft_plan_timing(plan.handle, int(bool(enable))))


def rsft_copy_buckets(plan: Plan, which: int, out, stream=None) -> None:
    _check(load_library().rsft_copy_buckets(plan.handle, int(which), _dptr(out, "out"), _stream(stream)))


def rsft_copy_detections(plan: Plan, out, stream=None) -> None:
    _check(load_library().rsft_copy_detections(plan.handle, _dptr(out, "out"), _stream(stream)))


def rsft_refine(plan: Plan, cube, k, freq, amp, steps, lr, stream=None) -> None:
    """Fold the cube, then `steps` Levenberg-Marquardt updates of the K tones in place
    (freq: device float32 [K, D] cycles/sample, amp: device complex64 [K])."""
    _check(load_library().rsft_refine(plan.handle, _dptr(cube, "cube"), int(k), _dptr(freq, "freq"),
                                      _dptr(amp, "amp"), int(steps),
                                      ctypes.c_float(lr), _stream(stream)))


def rsft_refine_prepare(plan: Plan, cube, stream=None) -> None:
    """Fold the cube into the plan's buckets (the data side of the refinement loss)."""
    _check(load_library().rsft_refine_prepare(plan.handle, _dptr(cube, "cube"), _stream(stream)))


def rsft_refine_eval(plan: Plan, freq, amp, loss=None, grad_freq=None, grad_amp=None, hdiag=None,
                     stream=None) -> None:
    """Loss (device float64 [1]), gradients (float32 [K, D], complex64 [K] holding (dE/da_re,
    dE/da_im)) and Gauss-Newton diagonal (float32 [K, D + 1]) of the tones."""
    k = int(amp.shape[0])
    _check(load_library().rsft_refine_eval(plan.handle, k, _dptr(freq, "freq"), _dptr(amp, "amp"),
                                           _dptr(loss, "loss"), _dptr(grad_freq, "grad_freq"),
                                           _dptr(grad_amp, "grad_amp"), _dptr(hdiag, "hdiag"), _stream(stream)))


def _check_stage2_tensors(votes, n, located, count, located_votes, cap):
    """Sizes, types and devices of rsft_stage2_static's tensors, checked before any launch: the C
    call sees only pointers, so a tensor shorter than n or cap would be read or written past its end."""
    given = [("votes", votes), ("count", count), ("located", located), ("located_votes", located_votes)]
    for what, t in given:
        if t is not None and not (hasattr(t, "is_cuda") and t.is_cuda):
            kind = "a CPU tensor" if hasattr(t, "is_cuda") else type(t).__name__
            raise TypeError(f"{what} must be a CUDA tensor (device memory), not {kind}")
    import torch
    dtypes = {"votes": (torch.uint8,), "count": (torch.int64,), "located_votes": (torch.uint8,),
              "located": (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ())}
    dev = torch.cuda.current_device()
    for what, t in given:
        if t is None:
            continue
        if t.dtype not in dtypes[what]:
            raise TypeError(f"{what} must have dtype {' or '.join(str(d) for d in dtypes[what])}, not {t.dtype}")
        if t.device.index != dev:
            raise ValueError(f"{what} must be on the current CUDA device (cuda:{dev})")
        if not t.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
    if int(n) > votes.numel():
        raise ValueError(f"n = {int(n)} exceeds the {votes.numel()} votes of the tensor")
    if count is None or count.numel() < 1:
        raise ValueError("count must hold at least one element")
    if cap < 0:
        raise ValueError("capacity must be >= 0")
    if cap > 0 and located is None:
        raise ValueError("located is required when capacity > 0")
    if located is not None and cap > located.numel():
        raise ValueError(f"capacity {cap} exceeds the {located.numel()} entries of located")
    if located_votes is not None and cap > located_votes.numel():
        raise ValueError(f"capacity {cap} exceeds the {located_votes.numel()} entries of located_votes")


def rsft_stage2_static(votes, n, mu, located, count, located_votes=None, capacity=None, stream=None) -> None:
    """Second-stage compaction into caller buffers, with library-owned fixed scratch
    (no device allocation); ``votes`` is cleared.  See include/rsft.h.

    Tensors are checked against n and the capacity before the call (ValueError / TypeError);
    the C entry point itself checks the limits it can see (alignment, n a multiple of 16384 and
    at most 2^28, mu)."""
    cap = (int(located.numel()) if located is not None else 0) if capacity is None else int(capacity)
    _check_stage2_tensors(votes, n, located, count, located_votes, cap)
    _check(load_library().rsft_stage2_static(_dptr(votes, "votes"), int(n), int(mu), _dptr(located, "located"),
                                             _dptr(located_votes, "located_votes"), cap, _dptr(count, "count"),
                                             _stream(stream)))


def rsft_check_wait_timeout(limit_ms: int = 20, stream=None) -> int:
    """Run the bounded-wait check; returns the status (RSFT_ERR_TIMEOUT is the expected one)."""
    return int(load_library().rsft_check_wait_timeout(int(limit_ms), _stream(stream)))


def rsft_status_string(status: int) -> str:
    return load_library().rsft_status_string(int(status)).decode()


def rsft_last_error() -> str:
    return load_library().rsft_last_error().decode()


class Graph:
    """Owning handle of an ``rsft_graph`` (one execute recorded as a CUDA graph); keeps its plan
    and the tensors whose pointers the graph holds alive."""

    def __init__(self, handle: c_void_p, plan: Plan, keep):
        self.handle = handle
        self.plan = plan
        self._keep = keep

    def launch(self, stream=None) -> None:
        _check(load_library().rsft_graph_launch(self.handle, _stream(stream)))

    def close(self):
        if self.handle:
            load_library().rsft_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rsft_graph_create(plan: Plan, cube, count, located=None, amp=None, lane: int = 0) -> Graph:
    """Record one execute of `plan` on `cube` (results to located / amp / count) on `lane`."""
    h = c_void_p()
    _check(load_library().rsft_graph_create(plan.handle, _dptr(cube, "cube"), int(lane), _dptr(located, "located"),
                                            _dptr(amp, "amp"), _dptr(count, "count"),
                                            ctypes.byref(h)))
    return Graph(h, plan, (cube, count, located, amp))


def rsft_graph_create_frames(plan: Plan, cubes, counts, located=None, amp=None) -> Graph:
    """Record rsft_execute_frames of `cubes` (results to located / amp / counts) as one CUDA graph."""
    h = c_void_p()
    _check(load_library().rsft_graph_create_frames(plan.handle, _dptr_array(cubes, "cubes"), len(cubes),
                                                   _dptr(located, "located"), _dptr(amp, "amp"),
                                                   _dptr(counts, "counts"), ctypes.byref(h)))
    return Graph(h, plan, (list(cubes), counts, located, amp))


def rsft_graph_launch_batch(graphs, stream=None) -> None:
    """Launch recorded executes (possibly of different plans), each lane's graphs in order."""
    arr = (c_void_p * max(1, len(graphs)))(*[g.handle for g in graphs])
    _check(load_library().rsft_graph_launch_batch(arr, len(graphs), _stream(stream)))


def rsft_plan_autotune(plan: Plan, cube, candidates: int = 4, reps: int = 10, stream=None):
    """Time the cost model's best `candidates` fold schedules on `cube`, keep the fastest.
    Returns (microseconds per fold launch of the winner, its rank among the candidates)."""
    us = ctypes.c_double(0.0)
    chosen = c_int32(-1)
    _check(load_library().rsft_plan_autotune(plan.handle, _dptr(cube, "cube"), _stream(stream), int(candidates),
                                             int(reps),
                                             ctypes.byref(us), ctypes.byref(chosen)))
    return float(us.value), int(chosen.value)


def rsft_plan_set_loops_per_pass(plan: Plan, loops_per_pass: int) -> None:
    """Fold `loops_per_pass` loops per pass over the cube (1..16)."""
    _check(load_library().rsft_plan_set_loops_per_pass(plan.handle, int(loops_per_pass)))


class BartlettPlan:
    """Owning handle of an ``rsft_bartlett_plan`` (the dense comparison detector)."""

    def __init__(self, handle: c_void_p, desc: RsftDesc):
        self.handle = handle
        self.desc = desc

    @property
    def shape(self):
        return tuple(int(self.desc.n[i]) for i in range(self.desc.ndim))

    def close(self):
        if self.handle:
            load_library().rsft_bartlett_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rsft_bartlett_plan_create(desc: RsftDesc) -> BartlettPlan:
    h = c_void_p()
    _check(load_library().rsft_bartlett_plan_create(ctypes.byref(desc), ctypes.byref(h)))
    return BartlettPlan(h, desc)


def rsft_bartlett_plan_destroy(plan: BartlettPlan) -> None:
    plan.close()


def rsft_bartlett_execute(plan: BartlettPlan, cube, located=None, amp=None, stream=None, allow_capacity=False) -> int:
    """Dense detection of a device cube; returns the number of detected bins."""
    n = c_int64(0)
    st = load_library().rsft_bartlett_execute(plan.handle, _dptr(cube, "cube"), _stream(stream),
                                              _dptr(located, "located"), _dptr(amp, "amp"),
                                              ctypes.byref(n))
    _check(st, allow=(RSFT_ERR_CAPACITY,) if allow_capacity else ())
    return int(n.value)


def rsft_bartlett_execute_async(plan: BartlettPlan, cube, count, located=None, amp=None, stream=None) -> None:
    _check(load_library().rsft_bartlett_execute_async(plan.handle, _dptr(cube, "cube"), _stream(stream),
                                                      _dptr(located, "located"), _dptr(amp, "amp"),
                                                      _dptr(count, "count")))


def rsft_bartlett_get(plan: BartlettPlan, what: int):
    if what == RSFT_BARTLETT_WINDOW:
        out = np.zeros(sum(plan.shape), dtype=np.float64)
    elif what == RSFT_BARTLETT_WORKSPACE_BYTES:
        out = np.zeros(1, dtype=np.int64)
    else:
        out = np.zeros(1, dtype=np.float64)
    _check(load_library().rsft_bartlett_get(plan.handle, what, out.ctypes.data_as(c_void_p), out.nbytes))
    return out


def rsft_bartlett_copy_spectrum(plan: BartlettPlan, out, stream=None) -> None:
    _check(load_library().rsft_bartlett_copy_spectrum(plan.handle, _dptr(out, "out"), _stream(stream)))
