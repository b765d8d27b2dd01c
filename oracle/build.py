"""Compile the CPU oracle (plain C, gcc, OpenMP) into oracle/_liboracle.so.

Test infrastructure only: the product path never loads this library.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hdd_oracle.c")
HDR = os.path.join(HERE, "hdd_oracle.h")
LIB = os.path.join(HERE, "_liboracle.so")


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in (SRC, HDR, __file__))


def build(force: bool = False) -> str:
    if force or needs_build():
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-D_DEFAULT_SOURCE", "-Wall", "-Wno-unknown-pragmas",
               SRC, "-o", LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
