"""Compile the CPU oracle (plain C, OpenMP when the compiler has it).

TEST INFRASTRUCTURE ONLY: the oracle library is used by the tests, the smoke
check and the benchmark's CPU baseline, never by the product path."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "spgemm_oracle.c"), os.path.join(HERE, "triangles_oracle.c")]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *SRCS, "-o", LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
