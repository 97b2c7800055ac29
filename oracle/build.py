"""Builds the oracle's shared library (liboracle.so) with the host C compiler.

Test infrastructure only: the oracle is compiled so the tests, the smoke check
and the CPU-baseline leg of the benchmark can call it.  Plain IEEE double
arithmetic: no fast-math, no FMA contraction, so x86 and Arm hosts agree;
OpenMP loops where the compiler offers it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["ionic.c", "fem.c", "sim.c"]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "oracle.h"), os.path.abspath(__file__)]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-Wall", "-Wextra"]
    # OpenMP when the compiler has it (the parallel loops' results do not
    # depend on the thread count); otherwise the same code runs on one thread
    r = subprocess.run(base + ["-fopenmp", "-o", LIB + ".tmp"] + srcs + ["-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base + ["-o", LIB + ".tmp"] + srcs + ["-lm"], check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
