"""Compile the oracle's C source into a shared library next to it.

Plain gcc, no vectoriser-dependent flags that change results:
-O2 -ffp-contract=off keeps every product and sum a separately rounded IEEE
operation except the explicit fma() calls.  The library is rebuilt when the
source is newer than it.  Portable C only (it builds on x86-64 and aarch64).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lc_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liblc_oracle.so")
OUT_OMP = os.path.join(OUT_DIR, "liblc_oracle_omp.so")


def build_oracle(force: bool = False, openmp: bool = False) -> str:
    """Build the serial parity oracle (default) or, with openmp=True, the
    timing-only OpenMP build of the same source (row loops in parallel, dot
    products as OpenMP reductions: other rounding, never used for parity)."""
    out = OUT_OMP if openmp else OUT
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall"] + (["-fopenmp"] if openmp else []) + ["-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
    print(build_oracle(force="--force" in sys.argv, openmp=True))
