"""Compile the CPU oracle (plain C) into oracle/liborc_apbf.so.

TEST INFRASTRUCTURE ONLY: the oracle is used by the tests, the smoke check and
the benchmark's CPU-baseline leg, never by the product path.

-ffp-contract=off matters: the oracle's FP32 decisions (cell index, neighbour
predicate, LOD level, prediction) must round after every operation, and gcc
contracts a*b+c into an FMA by default on aarch64.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "apbf_oracle.c")
HDR = os.path.join(HERE, "apbf_oracle.h")
LIB = os.path.join(HERE, "liborc_apbf.so")

CFLAGS = ["-O2", "-std=c11", "-Wall", "-Wextra", "-ffp-contract=off", "-fno-fast-math",
          "-fPIC", "-shared"]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in (SRC, HDR, __file__))


def build(force: bool = False) -> str:
    """Compile with OpenMP for the per-particle loops; a toolchain without it
    gets the same code compiled serially (the pragmas are then ignored)."""
    if force or needs_build():
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", *CFLAGS, "-fopenmp", SRC, "-o", tmp, "-lm"]
        if subprocess.run(cmd, stderr=subprocess.DEVNULL).returncode != 0:
            subprocess.run(["gcc", *CFLAGS, SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
