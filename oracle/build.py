"""Build the FP64 CPU oracle (test infrastructure) as a shared library.

Compiled with -ffp-contract=off so every floating-point operation rounds
once, and with OpenMP over the element and edge loops when the compiler
offers it.  Run as ``python oracle/build.py``; the test suite, the smoke
check and the benchmark's CPU-baseline leg call :func:`build` themselves.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lxw_oracle.c")
SRCS = [SRC, os.path.join(HERE, "lxw_oracle3d.c")]
HDRS = [os.path.join(HERE, "lxw_oracle.h"), os.path.join(HERE, "lxw_oracle3d.h")]
LIB = os.path.join(HERE, "liblxw_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in SRCS + HDRS):
        return LIB
    base = ["gcc", "-O3", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11", "-o", LIB + ".tmp"] + SRCS + ["-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
