"""Builds liblbm.so (the CUDA library behind include/lbm.h) in-tree for sm_103a.

Each translation unit compiles in parallel with nvcc; objects are reused when
they are newer than every source and header.  Output: _build/liblbm.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblbm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; liblbm needs the CUDA toolkit to build")
    return cand


def _deps():
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")))


def _compile(src: str, obj: str, ptxas_info: bool, extra=()) -> str:
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj + ".tmp"]
    if ptxas_info:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return r.stderr


def build(force: bool = False, ptxas_info: bool = False, jobs: int | None = None, checked: bool = False) -> str:
    """Compiles every csrc/*.cu and links _build/liblbm.so; returns its path.
    checked=True builds the bounds-checked library (LBM_BOUNDS_CHECK: every
    access of the step kernels checked against its plane, see
    lbm_bounds_check) into _build/checked/liblbm.so instead."""
    out = os.path.join(OUT, "checked") if checked else OUT
    lib = os.path.join(out, "liblbm.so")
    os.makedirs(out, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    dep_time = max(os.path.getmtime(p) for p in _deps() + srcs)
    todo = []
    objs = []
    for s in srcs:
        o = os.path.join(out, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or ptxas_info or not os.path.exists(o) or os.path.getmtime(o) < dep_time:
            todo.append((s, o))
    logs = []
    extra = ["-DLBM_BOUNDS_CHECK"] if checked else []
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for log in ex.map(lambda so: _compile(so[0], so[1], ptxas_info, extra), todo):
                logs.append(log)
    if todo or not os.path.exists(lib):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    if ptxas_info:
        sys.stderr.write("".join(logs))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, ptxas_info="-v" in sys.argv, checked="--checked" in sys.argv))
