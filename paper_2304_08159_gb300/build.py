"""Build libwl.so (the CUDA library behind include/wl.h) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into
paper_2304_08159_gb300/libwl.so.  No CMake; one -gencode.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwl.so")
# the bounds-checked build: the same sources with WL_DEBUG_BOUNDS (index checks that flag
# and skip, canaries between workspace arrays), for the tests
DEBUG_BUILD = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(HERE, "libwl_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra_flags=None, debug: bool = False) -> str:
    """Compile and link libwl.so (debug: the bounds-checked libwl_debug.so) if any source or
    header changed; return its path."""
    BUILD = DEBUG_BUILD if debug else globals()["BUILD"]
    LIB = DEBUG_LIB if debug else globals()["LIB"]
    if debug:
        extra_flags = list(extra_flags or []) + ["-DWL_DEBUG_BOUNDS"]
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "wl.h"))
    flags = FLAGS + list(extra_flags or [])
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if _stale(obj, [src] + headers):
            jobs.append([nvcc, *ARCH, *flags, "-c", src, "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(run, jobs))
    if jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


def build_all(verbose: bool = False):
    """Both libraries, compiled side by side."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        fs = [ex.submit(build, verbose), ex.submit(build, verbose, None, True)]
        return [f.result() for f in fs]


if __name__ == "__main__":
    print(build_all(verbose="-v" in sys.argv))
