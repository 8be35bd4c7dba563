"""Compile libxm.so (the CUDA library behind include/xm.h) for sm_103a, in-tree.

Run as ``python -m paper_2502_04640_b300.build`` or call ``build()``.  Each translation unit
is compiled by nvcc into ``_build/`` next to the sources, then linked into
``paper_2502_04640_b300/libxm.so`` (CUDA runtime only: no vendor math library).  Rebuilds only what is
older than its sources or headers.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libxm.so")
SOURCES = ["xm_api.cu", "xm_build.cu", "xm_qy.cu", "xm_qy_tc.cu", "xm_solver.cu", "xm_noalloc.cu", "xm_backward.cu",
           "xm_batched.cu", "xm_recover.cu", "xm_ozaki.cu", "xm_factored.cu", "xm_dense.cu", "xm_spdinv.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", INCLUDE]


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(INCLUDE, "xm.h"))
    return max(os.path.getmtime(h) for h in hdrs)


def _compile(src: str, extra: list, verbose: bool) -> str:
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    srcp = os.path.join(CSRC, src)
    if not extra and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(srcp), _deps()):
        return obj
    cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", srcp, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr.strip():
        print(res.stderr, flush=True)
    return obj


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, verbose or ptxas_info), SOURCES))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [NVCC, *ARCH, "-shared", "-o", LIB, *objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv))
