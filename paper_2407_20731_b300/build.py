"""Build libsemr.so in-tree with nvcc for sm_103a (B300), and its checking
variant libsemr_bounds.so (-DSEMR_BOUNDS: every kernel tests the index or byte
range of each global access against its buffer and skips, flagging
SEMR_STATUS_BOUNDS, any that falls outside)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libsemr.so")
LIB_BOUNDS = os.path.join(HERE, "libsemr_bounds.so")
SOURCES = [os.path.join(HERE, "csrc", s) for s in ("semr_kernels.cu", "semr_fast.cu", "semr_api.cpp", "semr_tables.cpp", "semr_noalloc.cu", "semr_batch.cpp", "semr_server.cpp", "semr_slice.cu", "semr_warp.cu", "semr_group.cu")]
HEADERS = [os.path.join(HERE, "csrc", h) for h in ("semr_internal.h", "semr_device.cuh", "semr_warp_common.cuh")] + [os.path.join(ROOT, "include", "semr.h")]

NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "-shared", "-cudart", "static"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in SOURCES + HEADERS)


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compile each source to an object under _build/ (in parallel), then link."""
    lib = LIB_BOUNDS if bounds else LIB
    if not (force or stale(lib)):
        return lib
    from concurrent.futures import ThreadPoolExecutor
    odir = os.path.join(ROOT, "_build", "bounds" if bounds else "default")
    os.makedirs(odir, exist_ok=True)
    cflags = [f for f in NVCC_FLAGS if f not in ("-shared", "-cudart", "static")]
    extra = (["-DSEMR_BOUNDS"] if bounds else []) + (["-Xptxas", "-v"] if verbose else [])

    def obj(src: str) -> str:
        o = os.path.join(odir, os.path.basename(src) + ".o")
        subprocess.run([nvcc()] + cflags + extra + ["-c", src, "-o", o], check=True)
        return o

    with ThreadPoolExecutor(min(len(SOURCES), os.cpu_count() or 1)) as ex:
        objs = list(ex.map(obj, SOURCES))
    subprocess.run([nvcc(), "-shared", "-cudart", "static", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-Xcompiler", "-fPIC"] + objs + ["-o", lib], check=True)
    return lib


def build_all(force: bool = False) -> None:
    """Both variants, compiled side by side."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(2) as ex:
        for r in [ex.submit(build, force, False, b) for b in (False, True)]:
            r.result()


if __name__ == "__main__":
    if "--bounds" in sys.argv:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds=True))
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
