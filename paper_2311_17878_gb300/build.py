"""Build ``libtsdfs.so`` (the C-ABI library) for sm_103a with nvcc, in-tree.

Each translation unit is compiled in parallel to ``_build/*.o`` and linked
into ``paper_2311_17878_gb300/libtsdfs.so``.  The fusion and bounds units are
compiled with ``--fmad=false`` (their results are bit-exact by contract).

    python -m paper_2311_17878_gb300.build [--force]
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
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libtsdfs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["abi.cu", "integrate.cu", "bounds.cu", "mlp_simt.cu", "composite.cu", "mlp_tc.cu", "mlp_pipe.cu", "backward.cu", "backward_gemm.cu", "fd64.cu"]
EXACT = {"integrate.cu", "bounds.cu"}


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hdrs + [os.path.join(INCLUDE, "tsdfs.h")]


def _compile(src, extra=()):
    s = os.path.join(CSRC, src)
    o = os.path.join(BUILD, src.replace(".cu", ".o"))
    newest = max(os.path.getmtime(p) for p in [s] + _deps())
    if os.path.exists(o) and os.path.getmtime(o) >= newest:
        return o, ""
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
           "-c", s, "-o", o + ".tmp", *extra]
    if src in EXACT:
        cmd.append("--fmad=false")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(o + ".tmp", o)
    return o, r.stderr


def build(force=False, verbose=False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            if f.endswith(".o"):
                os.remove(os.path.join(BUILD, f))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        res = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    objs = [o for o, _ in res]
    if verbose:
        for _, err in res:
            if err:
                print(err, file=sys.stderr)
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcuda", "-lcublas"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
