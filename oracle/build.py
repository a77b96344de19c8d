"""Builds the FP64 CPU oracle (test infrastructure) as a shared library.

Plain gcc, -O2, no fast-math, -ffp-contract=off so that the rounding does not
depend on whether the host has FMA.  OpenMP is used when the compiler has it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "admm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, quiet: bool = True) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC",
            "-o", LIB + ".tmp", SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=quiet)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=quiet)  # no OpenMP: serial
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, quiet=False))
