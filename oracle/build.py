"""Compile the FP64 CPU oracle (test infrastructure) into oracle/_build/.

Two builds of the same source: liborc.so (serial) and liborc_omp.so (OpenMP: the
column loop of a round shared among the host's cores, with the serial build's
results).  Plain gcc, no architecture-specific flags, so the same source builds on
the x86 development host and on the Arm GPU host.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rl0_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liborc.so")
LIB_OMP = os.path.join(OUT_DIR, "liborc_omp.so")


def _compile(out, extra):
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-fPIC", "-shared"] + extra + ["-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)


def build(force: bool = False, openmp: bool = False) -> str:
    """Path of the serial build (openmp=False) or the OpenMP build, compiled if stale."""
    os.makedirs(OUT_DIR, exist_ok=True)
    out = LIB_OMP if openmp else LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
        _compile(out, ["-fopenmp"] if openmp else ["-Wno-unknown-pragmas"])
    return out


def build_all(force: bool = False):
    return build(force), build(force, openmp=True)


if __name__ == "__main__":
    print(build_all(force=True))
