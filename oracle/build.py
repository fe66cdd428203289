"""Compile the FP64 CPU oracle (test infrastructure) into shared libraries.

Two builds of the same source: ``liborc.so`` (single thread) and
``liborc_omp.so`` (OpenMP ``parallel for`` over rows, same arithmetic).
Both use ``-ffp-contract=off`` so that no fused multiply-add changes the
rounding of the plain C expressions.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "tlb_oracle.c"), os.path.join(HERE, "tlb_droplets.c")]
FLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared", "-Wall"]


def lib_path(omp=False):
    return os.path.join(HERE, "liborc_omp.so" if omp else "liborc.so")


def build(force=False):
    outs = []
    for omp in (False, True):
        out = lib_path(omp)
        if force or not os.path.exists(out) or os.path.getmtime(out) < max(
            *(os.path.getmtime(s) for s in SRCS), os.path.getmtime(os.path.join(HERE, "tlb_oracle.h"))
        ):
            cmd = ["gcc", *FLAGS, *(["-fopenmp"] if omp else ["-Wno-unknown-pragmas"]), *SRCS, "-o", out + ".tmp", "-lm"]
            subprocess.check_call(cmd)
            os.replace(out + ".tmp", out)
        outs.append(out)
    return outs


if __name__ == "__main__":
    print("\n".join(build(force="--force" in sys.argv)))
