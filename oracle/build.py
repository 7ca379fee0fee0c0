"""Compile the CPU oracle (plain C, FP64, no fast-math, no FMA contraction)
and the multi-threaded (OpenMP) CPU baseline beside it.

Test infrastructure: builds oracle/_build/libgsr_oracle.so and
oracle/_build/libgsr_cpu_omp.so with gcc.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gsr_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libgsr_oracle.so")


OMP_SRC = os.path.join(HERE, "gsr_cpu_omp.c")
OMP_LIB = os.path.join(OUT_DIR, "libgsr_cpu_omp.so")


def _compile(src, lib, extra):
    if os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(src):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-fno-strict-aliasing"] + extra + ["-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Build the oracle (and the OpenMP CPU baseline beside it); returns the oracle."""
    if force:
        for lib in (LIB, OMP_LIB):
            if os.path.exists(lib):
                os.remove(lib)
    try:  # the OpenMP baseline is optional: a host without libgomp still builds the oracle
        _compile(OMP_SRC, OMP_LIB, ["-fopenmp"])
    except (subprocess.CalledProcessError, OSError) as e:
        sys.stderr.write("OpenMP CPU baseline not built: %s\n" % e)
    return _compile(SRC, LIB, [])


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
