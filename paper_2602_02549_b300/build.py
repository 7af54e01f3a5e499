"""Build liboz2.so (the C-ABI library) in-tree with nvcc for sm_103a.

    python -m paper_2602_02549_b300.build [--force] [-v]
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "liboz2.so")
SOURCES = [os.path.join(CSRC, "oz2_api.cu"), os.path.join(CSRC, "oz2_noalloc.cu"),
           os.path.join(CSRC, "oz2_tables.cpp")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    return SOURCES + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(CSRC, "*.cu")) + [os.path.join(INCLUDE, "oz2.h")]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in _inputs())
        if os.path.getmtime(LIB) >= newest:
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC,
           "-Xptxas", "-v" if verbose else "-O3", *SOURCES, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
