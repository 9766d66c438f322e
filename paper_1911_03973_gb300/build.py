"""Build libebe.so in-tree for sm_103a (GB300).

Each CUDA translation unit is compiled by nvcc in parallel, the host planner
by g++, then nvcc links the shared library next to this file.  No CMake.
Usage: ``python -m paper_1911_03973_gb300.build [--force]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libebe.so")

CU_SOURCES = ["k_patch.cu", "k_assemble.cu", "k_vec.cu", "k_batch.cu", "k_mpnn.cu", "k_alt.cu", "k_small.cu", "api.cu"]
CXX_SOURCES = ["plan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libebe.so")


def _sources_newer(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "ebe.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source for sm_103a and link ``libebe.so``; returns its path."""
    if not force and not _sources_newer(LIB):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-I", CSRC, "-I", INCLUDE]
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append([nvcc, *ARCH, *common, "-lineinfo", "-Xcompiler", "-fPIC", "-c", os.path.join(CSRC, src), "-o", obj])
    for src in CXX_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-I", CSRC, "-I", INCLUDE, "-c",
                     os.path.join(CSRC, src), "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(BUILD, s + ".o") for s in CU_SOURCES + CXX_SOURCES]
    tmp = LIB + f".tmp{os.getpid()}"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


def ptxas_report() -> str:
    """Registers / spills / shared memory per kernel (``-Xptxas -v``)."""
    nvcc = _nvcc()
    out = []
    for src in CU_SOURCES:
        out.append(_run([nvcc, *ARCH, "-O3", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-Xptxas", "-v", "-c",
                         os.path.join(CSRC, src), "-o", os.devnull]))
    return "\n".join(out)


if __name__ == "__main__":
    if "--ptxas" in sys.argv:
        print(ptxas_report())
    else:
        print(build(force="--force" in sys.argv, verbose=True))
