"""Builds the CUDA library ``_lib/libsdm.so`` in-tree for sm_103a.

One translation unit (``csrc/sdm_runtime.cu`` with the kernel headers),
compiled by nvcc for ``-gencode arch=compute_103a,code=sm_103a``.  Host code is
portable C++17 (the library builds unchanged on x86-64 and aarch64).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libsdm.so")
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "sdm.h")

GENCODE = "arch=compute_103a,code=sm_103a"
NVCC_FLAGS = [
    "-O3", "-lineinfo", "-std=c++17", f"-gencode={GENCODE}",
    "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr", "-cudart", "shared",
]


def sources():
    out = [HEADER]
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            out.append(os.path.join(CSRC, f))
    return out


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(LIB_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in sources()):
            return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc(), *NVCC_FLAGS, *extra, os.path.join(CSRC, "sdm_runtime.cu"), "-o", tmp]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else ()))
