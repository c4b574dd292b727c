"""Compile the plain FP64 CPU oracle (test infrastructure only).

The oracle is a checker: the test suite, the smoke check and the benchmark's
CPU-baseline leg load it; the product library never does.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pic_oracle.cpp")
LIB = os.environ.get("PIC_ORACLE_LIB") or os.path.join(HERE, "libpic_oracle.so")


def build(force: bool = False) -> str:
    """Build oracle/libpic_oracle.so with g++ (rounded as written: no FMA contraction)."""
    if os.environ.get("PIC_ORACLE_LIB"):
        return LIB  # a prebuilt oracle variant (used to check that the pins catch planted mistakes)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
