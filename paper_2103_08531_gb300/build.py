"""Build the solver's CUDA library (libfsp.so) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel into _build/, then linked
into paper_2103_08531_gb300/libfsp.so (CUDA runtime linked statically).  Runs
without a GPU: nvcc cross-compiles.  Rebuilds only when a source is newer than
the library, unless force=True.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfsp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfsp.so")
    return path


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _compile(src: str, extra: list[str], build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{res.stderr[-6000:]}")
    return obj


DEBUG_LIB = os.path.join(HERE, "libfsp_debug.so")


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          debug_bounds: bool = False) -> str:
    """Compile and link libfsp.so; returns its path.  debug_bounds=True builds
    libfsp_debug.so instead, with FSP_DEBUG_BOUNDS: every intermediate and grid
    index checked against its buffer (a bad one is recorded in the plan's device
    status and redirected, not faulted)."""
    lib = DEBUG_LIB if debug_bounds else LIB
    if not force and up_to_date(lib):
        return lib
    build_dir = BUILD + ("_debug" if debug_bounds else "")
    os.makedirs(build_dir, exist_ok=True)
    extra = list(extra or []) + (["-DFSP_DEBUG_BOUNDS"] if debug_bounds else [])
    if verbose:
        extra += ["-Xptxas", "-v"]
    srcs = sources()
    workers = max(1, min(len(srcs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lpthread", "-ldl", "-lrt"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr[-4000:]}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    import time
    t = time.time()
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv), f"{time.time() - t:.1f}s")
