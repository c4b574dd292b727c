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


LIB_THREADS = os.path.join(HERE, "libpic_oracle_threads.so")


def build(force: bool = False, threads: bool = False) -> str:
    """Build oracle/libpic_oracle.so with g++ (rounded as written: no FMA contraction).
    threads=True builds libpic_oracle_threads.so instead: the same source with
    -fopenmp, whose whole steps push the particles on all host cores (for timing
    the oracle on the host; the tests compare it with the serial build)."""
    if os.environ.get("PIC_ORACLE_LIB") and not threads:
        return LIB  # a prebuilt oracle variant (used to check that the pins catch planted mistakes)
    lib = LIB_THREADS if threads else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    cmd += (["-fopenmp"] if threads else []) + ["-o", tmp, SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, threads="--threads" in sys.argv))
