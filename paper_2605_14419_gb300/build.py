"""Builds the CUDA library in-tree: ``paper_2605_14419_gb300/libzsort.so``.

Two translation units in one nvcc call: the CUDA library (sm_103a only,
GB300) and the host-side autotuner.  Run as
``python -m paper_2605_14419_gb300.build``; ``__graft_entry__.build()`` calls
``build()``.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libzsort.so")
SOURCES = [os.path.join(CSRC, "zsort.cu"), os.path.join(CSRC, "zsort_tune.cpp")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in ("zsort_device.cuh", "zsort_tasks.cuh")] + [
    os.path.join(ROOT, "include", h) for h in ("zsort.h", "zsort_tune.h")]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *NVCC_FLAGS, "-o", tmp, *SOURCES]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
