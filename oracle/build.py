"""Builds the CPU oracle (test infrastructure only) into oracle/libromap_oracle.so.

The oracle is plain C compiled with -ffp-contract=off so that its FP32
sampler stage rounds every operation separately, on x86-64 and on AArch64
alike (GCC contracts a*b+c into FMA by default on AArch64).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "romap_oracle.c")
LIB = os.path.join(HERE, "libromap_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-Wno-unused-parameter", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
