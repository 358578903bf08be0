"""Compile the C oracle into ``oracle/liboracle.so`` (plain gcc, no GPU).

-ffp-contract=off keeps every a*b+c as two roundings unless the source writes
fma(); -O2 without -ffast-math keeps IEEE semantics.  -fopenmp (when the
compiler has it) runs independent block and row loops on all host cores.  No host-specific flags,
so the same source builds on x86-64 and aarch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sdsl_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", SRC, "-o", tmp, "-lm"]
    # block and row loops in parallel where the compiler has OpenMP (same
    # results: reductions stay serial); plain serial build otherwise
    r = subprocess.run(cmd[:-3] + ["-fopenmp"] + cmd[-3:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
