"""Builds libtreepm.so in-tree with nvcc for sm_103a (no cmake, no torch).

Translation units compile in parallel; the shared library links cuFFT.
Host code is compiled without floating-point contraction so that the tree
root (computed on the host) rounds the same way on x86-64 and aarch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libtreepm.so")
SOURCES = ["runtime.cu", "build.cu", "walk.cu", "pm.cu", "noalloc.cu", "batch.cu", "integrate.cu", "ewald.cu",
           "diagnostics.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Per-file flags.  The walk flushes FP32 denormals to zero: its operands
# (offsets, masses, r^-3 products) stay many orders of magnitude above the
# denormal range, and without the flag each rsqrt and division carries a
# denormal-handling path (measured 5% of the walk's time).
FILE_FLAGS = {"walk.cu": ["-ftz=true"]}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtreepm")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
                   "-I", INCLUDE, "-I", CSRC, *extra]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "treepm.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and not extra_flags and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OBJDIR, exist_ok=True)
    objs = []
    cmds = []
    for src in SOURCES:
        obj = os.path.join(OBJDIR, src.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([nvcc, *_flags(list(extra_flags) + FILE_FLAGS.get(src, [])), "-c", os.path.join(CSRC, src), "-o",
                     obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        list(ex.map(run, cmds))
    tmp = LIB + ".%d.tmp" % os.getpid()
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcufft"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True))
