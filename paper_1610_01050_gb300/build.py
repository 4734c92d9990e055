"""Build the RSFT CUDA library (librsft.so) in-tree for sm_103a.

Compiles the CUDA translation units and the host plan in parallel with nvcc /
g++ and links one shared library under ``paper_1610_01050_gb300/_lib``.  No
CMake, no torch extension machinery: the library exposes only the C ABI of
``include/rsft.h``.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT, "librsft.so")

CU_SOURCES = ["capi.cu", "fold.cu", "fold_tc.cu", "spectrum.cu", "votes.cu", "bartlett.cu", "refine.cu"]
CPP_SOURCES = ["plan_host.cpp"]
HEADERS = ["device.cuh", "tma.cuh", "plan_host.h", "fold_schedule.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the RSFT library needs the CUDA toolkit")
    return cand


def _cuda_include() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(_nvcc()))), "include")


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(ROOT, "include", "rsft.h")] + [os.path.join(CSRC, h) for h in HEADERS]
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    if verbose and res.stderr:
        print(res.stderr, flush=True)
    return res


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link librsft.so; returns its path.  Rebuilds only stale objects."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    jobs = []
    objs = []
    for s in CU_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT, s + ".o")
        objs.append(obj)
        if force or _stale(obj, src):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *inc, "-c", src, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    for s in CPP_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT, s + ".o")
        objs.append(obj)
        if force or _stale(obj, src):
            cxx = shutil.which("g++") or "c++"
            jobs.append([cxx, "-O2", "-std=c++17", "-fPIC", *inc, "-I", _cuda_include(), "-c", src, "-o", obj])
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for f in [ex.submit(_run, j, verbose) for j in jobs]:
            f.result()
    if jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        _run([nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lcufft"], verbose)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    path = build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(path)
