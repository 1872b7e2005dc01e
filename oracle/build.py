"""Builds the oracle's shared library (plain C, gcc).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline leg use the oracle.  OpenMP is used for the row-parallel application
of rotations when the compiler supports it; the arithmetic is compiled with
-ffp-contract=off so that x86 and aarch64 hosts round identically.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liborc.so")
SRC = os.path.join(HERE, "bgu_oracle.c")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", LIB + ".tmp", SRC, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
