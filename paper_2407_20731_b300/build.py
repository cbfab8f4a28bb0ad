"""Build libsemr.so in-tree with nvcc for sm_103a (B300)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libsemr.so")
SOURCES = [os.path.join(HERE, "csrc", s) for s in ("semr_kernels.cu", "semr_fast.cu", "semr_api.cpp", "semr_tables.cpp", "semr_noalloc.cu", "semr_batch.cpp", "semr_server.cpp", "semr_slice.cu", "semr_warp.cu", "semr_group.cu")]
HEADERS = [os.path.join(HERE, "csrc", h) for h in ("semr_internal.h", "semr_device.cuh", "semr_warp_common.cuh")] + [os.path.join(ROOT, "include", "semr.h")]

NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "-shared", "-cudart", "static"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in SOURCES + HEADERS)


def build(force: bool = False, verbose: bool = False) -> str:
    if force or stale():
        cmd = [nvcc()] + NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) + SOURCES + ["-o", LIB]
        subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
