"""Build the CPU oracle shared library (test infrastructure; see oracle/src/oracle.h).

Compiled with -ffp-contract=off so that every double operation is a single IEEE
operation on every host (x86-64 and AArch64 alike)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = ["arith.c", "ntt.c", "rng.c", "fft.c", "ckks.c", "lintrans.c", "poly.c", "bts.c", "softmax.c", "api.c"]
LIB = os.path.join(HERE, "liboracle.so")


def build(force=False, verbose=False):
    srcs = [os.path.join(HERE, "src", s) for s in SRC]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) < t for s in srcs + [os.path.join(HERE, "src", "oracle.h")]):
            return LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unused-function", "-Wno-maybe-uninitialized",
           "-o", LIB + ".tmp"] + srcs + ["-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="-f" in sys.argv, verbose=True))
