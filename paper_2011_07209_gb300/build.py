"""Build ``lib/libexx.so`` (the CUDA pair path) in-tree with nvcc for sm_103a.

Translation units are compiled in parallel; the host planner is compiled with
floating-point contraction off (its offset-membership and h^-1 arithmetic
decides integers and follows a fixed operation order).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libexx.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["kernels.cu", "api.cu", "noalloc.cu"]
CPP_SOURCES = ["plan.cpp"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA path cannot be built")


def _sources():
    return [os.path.join(SRC, f) for f in CU_SOURCES + CPP_SOURCES] + \
        [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))] + [os.path.join(INCLUDE, "exx.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nv = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-I", INCLUDE, "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off"]
    jobs = []
    for f in CU_SOURCES:
        obj = os.path.join(OUT_DIR, f + ".o")
        jobs.append([nv, *ARCH, *common, "-c", os.path.join(SRC, f), "-o", obj])
    for f in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, f + ".o")
        jobs.append([nv, *common, "-x", "c++", "-c", os.path.join(SRC, f), "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
        return p.stderr

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for msg in ex.map(run, jobs):
            if verbose and msg:
                print(msg, file=sys.stderr)
    objs = [os.path.join(OUT_DIR, f + ".o") for f in CU_SOURCES + CPP_SOURCES]
    tmp = LIB + f".tmp{os.getpid()}"
    run([nv, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
