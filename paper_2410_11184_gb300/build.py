"""Compile the CUDA library libhe_gb300.so in-tree for sm_103a (GB300).

Every translation unit is built with --fmad=false (device) and -ffp-contract=off (host) so
that each double operation of the encoder and of the scale bookkeeping is one IEEE
operation, as in the CPU reference."""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libhe_gb300.so")
SOURCES = ["he_kernels.cu", "he_host.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "--fmad=false", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
         "-diag-suppress", "177"]


def _nvcc():
    for p in ("/usr/local/cuda/bin/nvcc", "nvcc"):
        if os.path.sep not in p or os.path.exists(p):
            return p
    return "nvcc"


def build(force=False, verbose=False):
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "he_gb300.h"))
    if not force and os.path.exists(LIB) and all(os.path.getmtime(d) < os.path.getmtime(LIB) for d in deps):
        return LIB
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    objs = [os.path.join(bdir, os.path.basename(s) + ".o") for s in srcs]
    nv = _nvcc()
    cmds = [[nv] + ARCH + FLAGS + ["-c", s, "-o", o] for s, o in zip(srcs, objs)]

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
        return r.stderr

    with cf.ThreadPoolExecutor(len(cmds)) as ex:
        for err in ex.map(run, cmds):
            if verbose and err.strip():
                print(err)
    run([nv] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lcudart"])
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="-f" in sys.argv, verbose=True))
