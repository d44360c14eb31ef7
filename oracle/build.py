"""Build the CPU oracle shared libraries (test infrastructure only).

Three builds of the same sources:
  liboracle.so        plain FP64 (`real` = double), serial
  liboracle_flops.so  the same code with `real` counting every flop, used to
                      measure the algorithmic flops per grid point
  liboracle_omp.so    the plain code with its independent point loops on
                      several host threads (OpenMP); bitwise the serial results,
                      for the full-size checks and the timed CPU baseline.
All are compiled with -O2 -ffp-contract=off so the rounding sequence is the
one written in the source.  Portable flags only (the GPU hosts are aarch64).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["eos.cpp", "c2p.cpp", "fd.cpp", "ccz4.cpp", "mhd.cpp", "patch.cpp", "api.cpp", "mlp.cpp", "amr.cpp", "les.cpp"]
HEADERS = ["oracle.hpp", "real.hpp"]
FLAGS = ["-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall"]


def _outdated(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False):
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, h) for h in HEADERS] + [os.path.abspath(__file__)]
    outs = []
    jobs = []
    for name, extra in (("liboracle.so", []), ("liboracle_flops.so", ["-DORACLE_COUNT_FLOPS"]),
                        ("liboracle_omp.so", ["-fopenmp"])):
        out = os.path.join(HERE, name)
        outs.append(out)
        if _outdated(out, deps):
            tmp = out + ".tmp%d" % os.getpid()
            cmd = ["g++"] + FLAGS + extra + srcs + ["-o", tmp]
            if verbose:
                print(" ".join(cmd))
            jobs.append((subprocess.Popen(cmd), tmp, out))
    for p, tmp, out in jobs:
        if p.wait() != 0:
            raise RuntimeError("oracle build failed")
        os.replace(tmp, out)
    return outs


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
