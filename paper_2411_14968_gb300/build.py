"""Builds libskyline.so (the C-ABI library of include/skyline.h) in-tree with
nvcc for sm_103a: one object per .cu file compiled in parallel, then one
shared-library link against the static CUDA runtime.

Floating point: no --use_fast_math (denormals are kept, no flush-to-zero) and
--fmad=false, so every FP32 operation of the partition keys and scores is a
single correctly rounded IEEE operation.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libskyline.so")
SOURCES = ["sky_engine_w4r4.cu", "sky_engine_w8r4.cu", "sky_engine_w4r2.cu", "sky_engine_w8r2.cu", "sky_api.cu",
           "sky_dom.cu", "sky_engine.cu", "sky_prep.cu", "sky_pipeline.cu", "sky_prims.cu", "sky_probe.cu",
           "sky_rank.cu", "sky_serve.cu", "sky_static.cu", "sky_tune.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--fmad=false", "-Xcompiler", "-fPIC,-O2",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libskyline")


def _inputs():
    deps = [os.path.join(CSRC, s) for s in SOURCES]
    deps += [os.path.join(CSRC, "sky_internal.cuh"), os.path.join(CSRC, "sky_pipeline.cuh"),
             os.path.join(CSRC, "sky_engine_impl.cuh"),
             os.path.join(CSRC, "sky_serve.cuh"), os.path.join(ROOT, "include", "skyline.h"),
             os.path.join(ROOT, "include", "skyline_diag.h"),
             os.path.abspath(__file__)]
    return deps


def is_stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(p) > t for p in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the library if any source is newer than it; returns its path."""
    if not force and not is_stale():
        return LIB_PATH
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
