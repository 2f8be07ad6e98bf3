"""Build the sm_103a shared libraries in-tree with nvcc.

``_lib/librq.so``: every translation unit of the method under ``csrc/``,
compiled in parallel for ``-gencode arch=compute_103a,code=sm_103a`` and
linked into one shared object with a plain C ABI (``include/rq.h``).
``_lib/libpeak.so``: the arithmetic-pipe throughput probes the benchmark uses
as measured roofline denominators (``csrc/peak_probe.cu``).  No torch headers
are involved.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "librq.so")
PEAK_LIB = os.path.join(LIBDIR, "libpeak.so")
PEAK_SOURCE = "peak_probe.cu"
SOURCES = ["rq_context.cu", "rq_setup.cu", "rq_eval.cu", "rq_sweep.cu", "rq_target.cu", "rq_geometry.cu", "rq_tr.cpp", "rq_static.cu", "rq_batch.cu", "rq_sweep_df64.cu", "rq_hessian.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librq.so")


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PEAK_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(PEAK_LIB))
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "rq.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of ``librq.so``."""
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(objdir, src + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, "-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        objs = list(ex.map(compile_one, SOURCES + [PEAK_SOURCE]))
    for lib, parts in ((LIB, objs[:-1]), (PEAK_LIB, objs[-1:])):
        tmp = lib + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *parts]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
