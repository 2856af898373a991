"""Compile the CUDA library ``libsfseg.so`` for sm_103a, in-tree.

Each ``csrc/*.cu`` translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo`` and linked into
``_build/libsfseg.so`` (static CUDA runtime, no torch types).  The same
sources compiled with ``-DSFSEG_DEBUG`` give ``_build/libsfseg_debug.so``, the
bounds-checked build (both are compiled in one parallel pass).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libsfseg.so")
LIB_DEBUG = os.path.join(BUILD, "libsfseg_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _flags(verbose_ptxas: bool):
    f = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2",
         "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(sources, headers) -> bool:
    if not (os.path.exists(LIB) and os.path.exists(LIB_DEBUG)):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_DEBUG))
    return any(os.path.getmtime(p) > t for p in sources + headers + [__file__])


def build(force: bool = False, verbose_ptxas: bool = False, quiet: bool = True) -> str:
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                     + glob.glob(os.path.join(INCLUDE, "*.h")))
    if not force and not _stale(sources, headers):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    flags = _flags(verbose_ptxas)

    def compile_one(job):
        src, debug = job
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + (".debug.o" if debug else ".o"))
        cmd = [nvcc, *flags, *(["-DSFSEG_DEBUG"] if debug else []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if (verbose_ptxas or not quiet) and not debug:
            sys.stderr.write(r.stderr)
        return obj

    jobs = [(src, d) for d in (False, True) for src in sources]
    with ThreadPoolExecutor(max_workers=min(max(os.cpu_count() or 1, 2), len(jobs))) as ex:
        objs = list(ex.map(compile_one, jobs))
    for lib, part in ((LIB, objs[:len(sources)]), (LIB_DEBUG, objs[len(sources):])):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *part]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, quiet=False))
