"""Build the CUDA libraries in-tree for sm_103a: ``paper_2408_01470_b300/libsabr_lmm.so`` (the
calibration library behind include/sabr_lmm.h) and ``libsabr_peaks.so`` (the pipe-throughput probes
the benchmark's roofline divides by).

Usage: ``python -m paper_2408_01470_b300.build [--force] [--verbose]``.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsabr_lmm.so")
PEAKS_LIB = os.path.join(HERE, "libsabr_peaks.so")
PEAKS_SRC = os.path.join(CSRC, "peaks.cu")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def sources():
    return sorted([f for f in glob.glob(os.path.join(CSRC, "*.cu")) if f != PEAKS_SRC]
                  + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "sabr_lmm.h")])


def up_to_date(lib=LIB, srcs=None) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(s) <= t for s in (srcs or sources()))


def _compile(src, lib, verbose, extra):
    cmd = [NVCC, *ARCH, *FLAGS, *extra, src, "-o", lib + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if force or not up_to_date(PEAKS_LIB, [PEAKS_SRC]):
        _compile(PEAKS_SRC, PEAKS_LIB, verbose, ())
    if force or not up_to_date():
        _compile(os.path.join(CSRC, "api.cu"), LIB, verbose, extra)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB)
