"""Build the CUDA library libdts.so in-tree for sm_103a (B300).

Each translation unit under csrc/ is compiled to an object in _build/ (in
parallel), then linked into paper_1910_11335_b300/libdts.so. With
--debug-bounds the same sources are compiled with -DDTS_DEBUG_BOUNDS into
_build/debug/ and linked into libdts_debug.so (the bounds-checked build that
DTS_DEBUG_BOUNDS=1 makes the binding load).

    python -m paper_1910_11335_b300.build [--force] [--verbose] [--debug-bounds]
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libdts.so")
LIB_DEBUG = os.path.join(PKG, "libdts_debug.so")
OBJ = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps():
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        sorted(glob.glob(os.path.join(CSRC, "*.h"))) + \
        [os.path.join(ROOT, "include", "dts.h"), os.path.abspath(__file__)]


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps())


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    lib = LIB_DEBUG if debug_bounds else LIB
    if not force and not stale(lib):
        return lib
    obj_dir = os.path.join(OBJ, "debug") if debug_bounds else OBJ
    os.makedirs(obj_dir, exist_ok=True)
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
             "-I", os.path.join(ROOT, "include")]
    if debug_bounds:
        flags.append("-DDTS_DEBUG_BOUNDS")
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        subprocess.check_call([nvcc(), *flags, "-c", "-o", obj, src])
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(sources()), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", lib + ".tmp", *objs])
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
                debug_bounds="--debug-bounds" in sys.argv))
