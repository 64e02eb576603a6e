"""Builds the CUDA library libhot.so in-tree with nvcc for sm_103a (GB300)."""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libhot.so")
SOURCES = [os.path.join(CSRC, f) for f in ("hot.cu", "tc.cu", "once.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in ("gsw_kernels.cuh", "tc_kernels.cuh", "tc.h", "once.h")] + \
    [os.path.join(ROOT, "include", "hot.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhot.so")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of libhot.so."""
    if not force and up_to_date():
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    # the translation units compile in parallel, then link into one shared library
    objs = [f"{tmp}.{i}.o" for i in range(len(SOURCES))]
    procs = [subprocess.Popen([nvcc(), *flags, "-c", src, "-o", obj], stdout=subprocess.PIPE,
                              stderr=subprocess.STDOUT, text=True) for src, obj in zip(SOURCES, objs)]
    outs = [p.communicate()[0] for p in procs]
    try:
        for p, src, out in zip(procs, SOURCES, outs):
            if p.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{out}")
        link = [nvcc(), *ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + " ".join(link) + "\n" + r.stdout + r.stderr)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    if verbose:
        print("".join(outs))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
