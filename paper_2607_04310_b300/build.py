"""Builds libpsdf_b300.so (all CUDA sources in csrc/) for sm_103a, in-tree.

    python -m paper_2607_04310_b300.build [--force]

nvcc cross-compiles without a GPU.  Objects are compiled in parallel into
``_build/`` and linked into ``paper_2607_04310_b300/libpsdf_b300.so``.  A second
library, ``libpsdf_b300_debug.so``, links the same objects except the batched
kernels, which are compiled again with PSDF_DEBUG_CHECKS (every index they
take from their data checked, the first violation recorded); the tests load
it in a process of its own (PSDF_LIBRARY).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libpsdf_b300.so")
LIB_DEBUG = os.path.join(HERE, "libpsdf_b300_debug.so")
DEBUG_SOURCES = ("batched.cu",)  # compiled again with the index checks

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(ROOT, "include", "*.h")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run_jobs(jobs, verbose):
    if not jobs:
        return
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)


def _link(nvcc, objs, lib, force):
    if force or _stale(lib, objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False) -> str:
    """Both libraries, recompiling what is stale; returns the release path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    hdrs = headers()
    nvcc = _nvcc()
    objs, dobjs, jobs = [], [], []
    for src in srcs:
        obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            jobs.append([nvcc] + ARCH + NVCC_FLAGS + ["-c", src, "-o", obj])
        if os.path.basename(src) in DEBUG_SOURCES:
            dobj = obj.replace(".o", ".debug.o")
            dobjs.append(dobj)
            if force or _stale(dobj, [src] + hdrs):
                jobs.append([nvcc] + ARCH + NVCC_FLAGS + ["-DPSDF_DEBUG_CHECKS", "-c", src, "-o",
                                                          dobj])
        else:
            dobjs.append(obj)
    _run_jobs(jobs, verbose)
    _link(nvcc, objs, LIB, force or bool(jobs))
    _link(nvcc, dobjs, LIB_DEBUG, force or bool(jobs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
