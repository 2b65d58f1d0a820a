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
# one translation unit per kernel family, compiled in parallel and linked into one library
SOURCES = [os.path.join(SRC, f) for f in ("nvdb.cu", "eval_f32.cu", "eval_f16.cu", "eval_bf16.cu", "eval_bf16x3.cu",
                                          "eval_fp8.cu", "train_tc.cu", "calib.cu", "sort.cu")]
OBJDIR = os.path.join(HERE, "_build")


def _deps():
    return SOURCES + [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cuh", ".cu"))] + [
        os.path.join(ROOT, "include", "nvdb.h")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


FLAGS = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-gencode", "arch=compute_103a,code=sm_103a",
         "-lineinfo"]


def compile_command(src: str, obj: str, extra=()) -> list:
    return [nvcc(), *FLAGS, "-I", os.path.join(ROOT, "include"), "-c", "-o", obj, *extra, src]


def link_command(objs, out: str = LIB) -> list:
    return [nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", out, *objs]


def command(out: str = LIB, extra=()) -> list:
    """Single-step build of every unit (same flags as the parallel build)."""
    return [nvcc(), *FLAGS, "-shared", "-I", os.path.join(ROOT, "include"), "-o", out, *extra, *SOURCES]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _obj(src: str) -> str:
    return os.path.join(OBJDIR, os.path.basename(src)[:-3] + ".o")


def _headers_mtime() -> float:
    hs = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cuh")] + [os.path.join(ROOT, "include", "nvdb.h")]
    return max(os.path.getmtime(h) for h in hs)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    os.makedirs(OBJDIR, exist_ok=True)
    hdr = _headers_mtime()
    jobs = []
    for s in SOURCES:
        o = _obj(s)
        if force or extra or not os.path.exists(o) or os.path.getmtime(o) < max(hdr, os.path.getmtime(s)):
            jobs.append(compile_command(s, o + ".tmp", extra))

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(cmd[cmd.index("-o") + 1], cmd[cmd.index("-o") + 1][:-4])

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(run, jobs))
    tmp = LIB + ".tmp"
    cmd = link_command([_obj(s) for s in SOURCES], tmp)
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
