"""Builds libnufft3d.so in-tree with nvcc for sm_103a (no CMake, no torch).

Each .cu translation unit is compiled in parallel, then linked into a shared
library next to this file.  Object files go to <repo>/_build/ (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libnufft3d.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["plan.cu", "fft_passes.cu", "interp_gather.cu", "interp_spread.cu", "interp_tma.cu", "interp_real.cu", "noalloc.cu", "polar_nufft.cu", "grangeat.cu",
           "batch.cu", "polar_resample.cu", "peak.cu",
           "host_pipeline.cu"]
# nvcc's whole-TU code generation (--split-compile=0) schedules the gather
# kernels better and the shared-atomic spread kernels worse (both measured with
# CUDA events at 256^3), so it is applied per translation unit.
NO_SPLIT_COMPILE = {"interp_spread.cu"}


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnufft3d")


def _flags(src: str, extra=()):
    split = [] if src in NO_SPLIT_COMPILE or os.environ.get("NUFFT3D_SPLIT_COMPILE", "1") == "0" \
        else ["--split-compile=0"]
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", *split, "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
                   "-I", os.path.join(ROOT, "include"), *extra]


def _compile(src: str, extra=()) -> str:
    obj = os.path.join(BUILD, os.path.splitext(os.path.basename(src))[0] + ".o")
    cmd = [nvcc_path(), *_flags(src, extra), "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and (r.returncode < 0 or "Segmentation fault" in r.stdout + r.stderr):
        # a crashed compiler process (not a diagnostic): run it once more
        r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src} (exit {r.returncode}):\n{r.stdout}\n{r.stderr}")
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "nufft3d.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile every CUDA source for sm_103a and link libnufft3d.so."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc_path(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
