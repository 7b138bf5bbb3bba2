"""Builds the CUDA library ``_build/liblf.so`` in-tree for sm_103a.

One nvcc invocation per translation unit, run in parallel, then one link.
The library is a plain shared object with a C ABI (``include/lf.h``); the
Python binding loads it with ctypes.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblf.so")
# Test build with every step-kernel index checked against its array (-DLF_CHECKED).
LIB_CHECKED = os.path.join(BUILD, "liblf_checked.so")
SOURCES = ["lf_kernels.cu", "lf_lloyd.cu", "lf_dual.cu", "lf_cotan.cu", "lf_host.cpp", "lf_noalloc.cu",
           "lf_server.cpp"]
HEADERS = [os.path.join(CSRC, "lf_internal.h"), os.path.join(ROOT, "include", "lf.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-Wall,-pthread,-ffp-contract=off", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, checked=False):
    """Builds liblf.so, or with checked=True the bounds-checked test variant."""
    lib = LIB_CHECKED if checked else LIB
    objdir = os.path.join(BUILD, "checked") if checked else BUILD
    extra = ["-DLF_CHECKED"] if checked else []
    os.makedirs(objdir, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    if not force and not _stale(lib, srcs + HEADERS + [__file__]):
        return lib
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
