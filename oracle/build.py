"""Compile the oracle's C stepper into oracle/liboracle_d2q37.so and its instrumented flop
counter into oracle/count_collide_flops (test infrastructure only).

Plain gcc/g++, -O2 (-O0 for the counter), OpenMP, and -ffp-contract=off so that the oracle never
fuses a product into an addition on any host (x86_64 or aarch64). No machine-specific flags.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "d2q37_oracle.c")
LIB = os.path.join(HERE, "liboracle_d2q37.so")
COUNTER_SRC = os.path.join(HERE, "count_collide_flops.cpp")
COUNTER = os.path.join(HERE, "count_collide_flops")


def build_counter(force: bool = False) -> str:
    """Build the instrumented flop counter if it is missing or older than its sources."""
    newest = max(os.path.getmtime(SRC), os.path.getmtime(COUNTER_SRC))
    if not force and os.path.exists(COUNTER) and os.path.getmtime(COUNTER) >= newest:
        return COUNTER
    tmp = COUNTER + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O0", "-std=c++17", "-ffp-contract=off", "-I", HERE, "-o", tmp, COUNTER_SRC],
                   check=True)
    os.replace(tmp, COUNTER)
    return COUNTER


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_counter(force="--force" in sys.argv))
