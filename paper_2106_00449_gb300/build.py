"""Build the CUDA library libgdc.so in-tree for sm_103a (one -gencode, parallel nvcc)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgdc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "geometry.cu", "rpy.cu", "sym.cu", "body.cu", "krylov.cu", "cells.cu", "fcm.cu", "wall.cu", "dfsym.cu", "probe.cu"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the gDC library needs the CUDA toolkit to build")
    return exe


# the pair kernels flush FP32 denormals (their operands are never denormal), which lets
# rsqrtf map to the bare reciprocal-square-root unit operation; so do the FCM kernels (their
# Gaussians are 2^x with -21 < x <= 0 and their grid values are far from the denormal range),
# where it lets exp2f map to the bare exponential unit operation
PER_FILE = {"rpy.cu": ["-ftz=true"], "sym.cu": ["-ftz=true"], "fcm.cu": ["-ftz=true"]}


def _compile(src: str, extra) -> str:
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-lineinfo", "-std=c++17",
           "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", *ARCH, *PER_FILE.get(src, []), *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, list(extra)), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp, *objs, *ARCH, "-cudart", "shared"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
