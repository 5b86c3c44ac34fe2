"""Builds the in-tree shared library ``libtac.so`` (sm_103a) with nvcc.

Usage: ``python -m paper_2603_28475_b300.build [--verbose-ptxas]``.
The library has a plain C ABI (include/tac.h); the Python binding loads it
with ctypes.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = [os.path.join(PKG, "csrc", f) for f in ("kernels.cu", "kernels_wide.cu", "api.cu", "mesh.cpp")]
DEPS = SRC + [os.path.join(PKG, "csrc", f) for f in ("device_math.cuh", "solve.cuh", "mesh.h", "layout.h")] + \
    [os.path.join(ROOT, "include", "tac.h")]
LIB = os.path.join(PKG, "libtac.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force=False, ptxas_verbose=False):
    if not force and up_to_date():
        return LIB
    cmd = [nvcc(), "-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-o", LIB] + SRC
    if ptxas_verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if ptxas_verbose:
        sys.stdout.write(res.stdout + res.stderr)
    return LIB


if __name__ == "__main__":
    build(force=True, ptxas_verbose="--verbose-ptxas" in sys.argv)
    print(LIB)
