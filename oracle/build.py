"""Compile the CPU oracle (test infrastructure) into oracle/libspin_oracle.so,
and its all-cores sweep for the CPU baseline into oracle/libspin_oracle_omp.so
(the serial oracle plus spin_oracle_omp.c, built with OpenMP).

Plain gcc, ISO C11, no fast-math and no floating-point contraction, so the
double-precision threshold tables are the IEEE results of exp() and floor().
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spin_oracle.c")
LIB = os.path.join(HERE, "libspin_oracle.so")
OMP_SRC = os.path.join(HERE, "spin_oracle_omp.c")
OMP_LIB = os.path.join(HERE, "libspin_oracle_omp.so")
FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-Wall", "-Wextra", "-fPIC", "-shared"]


def _stale(lib, srcs):
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(f) for f in srcs)


# Several processes (the ranks of a multi-process test) may build at the
# same time: each writes its own temporary file and renames it into place.
def _tmp(lib):
    return f"{lib}.{os.getpid()}.tmp"


def build(force: bool = False) -> str:
    if force or _stale(LIB, [SRC]):
        tmp = _tmp(LIB)
        subprocess.run(["gcc", *FLAGS, SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


def build_omp(force: bool = False) -> str:
    if force or _stale(OMP_LIB, [SRC, OMP_SRC]):
        tmp = _tmp(OMP_LIB)
        subprocess.run(["gcc", *FLAGS, "-fopenmp", SRC, OMP_SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, OMP_LIB)
    return OMP_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_omp(force="--force" in sys.argv))
