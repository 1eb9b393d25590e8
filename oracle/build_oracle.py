"""Compile the FP64 CPU oracle (oracle.c) into oracle/_build/liboracle.so,
and its timing build (the per-agent force loop parallel over the host's
cores with OpenMP, each agent's sum still serial, so the results are the
same bits) into oracle/_build/liboracle_omp.so.

Test infrastructure: the oracle is used by the test suite, the smoke check and
the benchmark's CPU-baseline leg only.  -ffp-contract=off keeps every a*b+c
as two rounded operations (aarch64 GCC would otherwise fuse them).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall"]


def _compile(lib, extra, force):
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [os.environ.get("CC", "cc")] + CFLAGS + extra + [SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    return _compile(LIB, [], force)


def build_omp(force: bool = False):
    """The OpenMP timing build, or None where the compiler has no OpenMP."""
    try:
        return _compile(LIB_OMP, ["-fopenmp", "-DORC_OPENMP"], force)
    except (subprocess.CalledProcessError, OSError):
        return None


if __name__ == "__main__":
    print(build(force="--force" in sys.argv), build_omp(force="--force" in sys.argv))
