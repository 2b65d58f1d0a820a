"""Compile libnvdb.so in-tree for B300 (sm_103a) with nvcc.

    python -m paper_2208_04448_b300._build [--force]
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libnvdb.so")
SOURCES = [os.path.join(SRC, "nvdb.cu")]


def _deps():
    return SOURCES + [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cuh", ".cu"))] + [
        os.path.join(ROOT, "include", "nvdb.h")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def command(out: str = LIB, extra=()) -> list:
    return [nvcc(), "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC,-ffp-contract=off",
            "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
            "-I", os.path.join(ROOT, "include"), "-o", out, *extra, *SOURCES]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if force or not up_to_date():
        tmp = LIB + ".tmp"
        cmd = command(tmp)
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
