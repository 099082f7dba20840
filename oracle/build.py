"""Compile the oracle's C source into ``oracle/_build/liboracle.so`` with gcc.

Plain -O2 without fast-math and without floating-point contraction, so the
arithmetic is IEEE round-to-nearest double in the order written. With
openmp=True the same source is built with -fopenmp into liboracle_omp.so
(its node loops run on all host cores, with the same results bit for bit);
that build serves only the all-cores CPU baseline.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    lib = LIB_OMP if openmp else LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(SRC)):
        return lib
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11"] + (["-fopenmp"] if openmp else []) + ["-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
