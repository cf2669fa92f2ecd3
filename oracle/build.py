"""Build the oracle shared library (test infrastructure only).

The oracle is plain C++ compiled with the host compiler.  Floating-point
contraction is disabled so that binary32/binary64 operations happen exactly
as written (aarch64 GCC would otherwise fuse multiply-adds).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["oracle_physics.cpp", "oracle_transport.cpp", "oracle_scatter.cpp"]
LIB = os.path.join(HERE, "liboracle.so")


LIB_OMP = os.path.join(HERE, "liboracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """liboracle.so (the oracle); openmp=True builds liboracle_omp.so, the same
    source with the transport's cell loop spread over threads, used only to
    time the oracle on all host cores."""
    lib = LIB_OMP if openmp else LIB
    srcs = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, "oracle.h")]
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return lib
    extra = ["-fopenmp", "-DORACLE_OPENMP"] if openmp else []
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wextra"] + extra + ["-o", lib + ".tmp"] + [os.path.join(HERE, s) for s in SOURCES]
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build(force="--force" in sys.argv, openmp=True))
