"""Compile the C oracle (test infrastructure) into oracle/_build/liboracle.so.

The discrete path relies on an explicit float32 operation order, so the file
is built with -ffp-contract=off and without fast-math.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "psi_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False, verbose: bool = False, plant: int = 0) -> str:
    """Build the oracle; ``plant`` > 0 builds a deliberately wrong variant
    (used only by the test that checks the pins catch mistakes)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    lib = LIB if plant == 0 else os.path.join(OUT_DIR, f"liboracle_plant{plant}.so")
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wno-unknown-pragmas", f"-DOR_PLANT={int(plant)}", SRC, "-o", tmp, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
