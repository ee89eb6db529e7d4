"""Build libnpfem.so (the C-ABI CUDA library) in-tree for sm_103a.

Plain nvcc, no cmake: the translation units are compiled in parallel and
linked into ``paper_1911_03062_gb300/libnpfem.so``; the arithmetic-throughput
probes of the benchmark's peaks leg go into ``libnpfem_peaks.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libnpfem.so")
PEAKS_LIB = os.path.join(HERE, "libnpfem_peaks.so")
BUILD = os.path.join(ROOT, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-prec-div=false", "-prec-sqrt=false", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
SOURCES = ["npfem.cu"]
PEAKS_SOURCES = ["peaks.cu"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libnpfem.so")
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "npfem.h"))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    dep = _deps()
    if not force and all(os.path.exists(p) and os.path.getmtime(p) >= dep for p in (LIB, PEAKS_LIB)):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *NVFLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        return obj

    srcs = SOURCES + PEAKS_SOURCES
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    for lib, o in ((LIB, objs[:len(SOURCES)]), (PEAKS_LIB, objs[len(SOURCES):])):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *o])
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
