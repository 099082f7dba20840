"""Build the CUDA library ``_build/liblbm.so`` for sm_103a with nvcc.

Three translation units (the C ABI with its kernels, the TMA-staged step's
instantiations, and the allocation-free reduction), compiled in parallel
to objects and linked; one -gencode, in-tree output.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm.so")
SOURCES = [os.path.join(CSRC, "lbm_api.cu"), os.path.join(CSRC, "lbm_step_tma.cu"),
           os.path.join(CSRC, "lbm_noalloc.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + \
    [os.path.join(INCLUDE, "lbm.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def flags(extra=()):
    return ["-O3", "-lineinfo", ARCH, "-std=c++17", "-Xcompiler", "-fPIC",
            "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, *extra]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    extra = ["-Xptxas", "-v"] if verbose else []
    objs = [os.path.join(OUT_DIR, os.path.basename(src) + ".%d.o" % os.getpid()) for src in SOURCES]
    procs = [subprocess.Popen([nvcc(), "-c", *flags(extra), "-o", obj, src])
             for src, obj in zip(SOURCES, objs)]
    failed = [src for src, pr in zip(SOURCES, procs) if pr.wait() != 0]
    try:
        if failed:
            raise subprocess.CalledProcessError(1, "nvcc -c " + " ".join(failed))
        subprocess.run([nvcc(), "-shared", ARCH, "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
