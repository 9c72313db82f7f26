"""Compile the CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain C, OpenMP over independent gates/rows.  Floating point is used only
for key/noise sampling; it is compiled without fast-math or contraction so
that the Box-Muller values are the host libm's exact ones.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tfhe_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O3", "-fopenmp", "-fPIC", "-shared", "-fvisibility=hidden",
           "-fno-fast-math", "-ffp-contract=off", "-Wall", "-Wextra", "-Wno-unused-parameter",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
