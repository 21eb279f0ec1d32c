"""Build and load libclod (the sm_103a CUDA library behind include/clod.h).

The library is compiled in-tree with nvcc into ``paper_2510_09997_gb300/_build``
and loaded with ctypes.  There is no fallback: if the library cannot be built
or loaded, every entry point raises.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import glob
import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libclod.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
           "-Xcompiler", "-ffp-contract=off"]
# Translation units whose arithmetic decides nothing bit-exact outside the
# explicit round-to-nearest intrinsics may let nvcc fuse multiply-adds.
FMAD_OK = {"backward.cu", "loss.cu"}

_lock = threading.Lock()
_lib = None


def nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: libclod needs the CUDA toolkit to build")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in parallel, then link the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and not stale():
        return LIB
    nv = nvcc()
    srcs = _sources()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        flags = list(NVFLAGS)
        if os.path.basename(src) in FMAD_OK:
            flags[flags.index("--fmad=false")] = "--fmad=true"
        cmd = [nv, *ARCH, *flags, "-I", INCLUDE, "-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nv, *NVFLAGS, "-I", INCLUDE, "-x", "cu", *ARCH, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp.%d" % os.getpid()
    r = subprocess.run([nv, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


def load():
    """Load libclod (building it first if needed) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if stale():
            build()
        L = ctypes.CDLL(LIB)
        from . import abi
        abi.declare(L)
        _lib = L
        return L
