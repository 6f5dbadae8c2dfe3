"""Builds the CPU oracle (test infrastructure) as a shared library.

Compiled with ``-O2 -ffp-contract=off`` and no fast-math so that every
floating-point operation is one IEEE round-to-nearest step, as on the GPU side.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cbt_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcbt_oracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "cbt_oracle.h"))):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-Wall", "-fPIC",
                           "-shared", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
