"""In-tree build of the native parts: librst.so (CUDA, sm_103a) and the input generator.

The CUDA sources are compiled one translation unit per nvcc process, in
parallel, then linked into paper_2603_11645_gb300/librst.so.  Only the
sm_103a target is generated.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librst.so")
GEN_SRC = os.path.join(HERE, "gen", "graphgen.c")
GEN_LIB = os.path.join(HERE, "gen", "libgraphgen.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
           "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r


def build_generator() -> str:
    _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-pthread", "-D_DEFAULT_SOURCE",
          GEN_SRC, "-o", GEN_LIB, "-lpthread"])
    return GEN_LIB


def build_library(verbose_ptx: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    extra = ["-Xptxas", "-v"] if verbose_ptx else []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        r = _run([NVCC, *ARCH, *NVFLAGS, *extra, "-c", src, "-o", obj])
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    if verbose_ptx:
        for o, err in results:
            print(f"== {os.path.basename(o)}\n{err}")
    tmp = LIB + ".tmp"
    _run([NVCC, *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    build_generator()
    print(build_library(verbose_ptx="-v" in sys.argv))
