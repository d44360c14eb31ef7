"""Build libgrmhd.so (the CUDA kernels + C ABI) for sm_103a, in-tree.

Each .cu file is compiled in parallel with nvcc, then linked into
paper_2510_13965_gb300/libgrmhd.so.  Objects go to paper_2510_13965_gb300/_build/.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgrmhd.so")
SOURCES = ["api.cu", "kernels.cu", "rhs.cu", "noalloc.cu", "seeder.cu", "amr.cu", "les.cu", "shard.cu"]
HEADERS = ["dev.cuh", "c2p.cuh", "kern.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"] + ARCH


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps():
    inc = os.path.join(os.path.dirname(HERE), "include", "grmhd.h")
    return [os.path.join(CSRC, h) for h in HEADERS] + [inc, os.path.abspath(__file__)]


def build(verbose=False, ptxas_info=False):
    os.makedirs(BUILD, exist_ok=True)
    deps = _deps()
    nvcc = _nvcc()
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if not os.path.exists(o) or any(os.path.getmtime(d) > os.path.getmtime(o) for d in deps + [s]):
            cmd = [nvcc] + NVCC_FLAGS + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", s, "-o", o + ".tmp"]
            if verbose:
                print(" ".join(cmd), flush=True)
            jobs.append((subprocess.Popen(cmd), o))
    for p, o in jobs:
        if p.wait() != 0:
            raise RuntimeError("nvcc failed for " + o)
        os.replace(o + ".tmp", o)
    if not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lcudart"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv)
