"""Compile the oracle's C source with gcc: oracle/_build/liboracle.so (the
plain single-threaded oracle) and oracle/_build/liboracle_omp.so (the same
source with -fopenmp: its Jacobi-PCG shares the cell loops among the host
cores).

Test infrastructure: only the tests, the smoke check and the benchmark's
CPU-baseline and reference-solution legs load the results.
-ffp-contract=off keeps a*b+c unfused on every host so x86 and Arm builds
round alike.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ldu_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")


def library_path(omp=False):
    return LIB_OMP if omp else LIB


def needs_build(omp=False):
    lib = library_path(omp)
    return (not os.path.exists(lib)) or os.path.getmtime(lib) < os.path.getmtime(SRC)


def build(force=False, verbose=False, omp=False):
    lib = library_path(omp)
    if not force and not needs_build(omp):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", "-Wextra"] + (["-fopenmp"] if omp else []) + ["-o", tmp, SRC, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build_all(force=False, verbose=False):
    return [build(force, verbose, omp) for omp in (False, True)]


if __name__ == "__main__":
    print(build_all(force=True, verbose=True))
