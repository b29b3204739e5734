"""Builds the in-tree CUDA library ``libiffd.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared
library next to this file. Usage: ``python -m paper_2512_20269_gb300.build``
or ``build()`` from Python.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libiffd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["host_setup.cpp", "precond.cu", "precond_warp64.cu", "precond_warp128.cu", "precond_warp256.cu",
           "precond_warp512.cu", "precond_wdf64.cu", "precond_wdf128.cu", "precond_wdf256.cu", "stiffness.cu", "pcg.cu", "fd.cu", "capi.cu", "noalloc.cu", "varcoef.cu", "engine.cu",
           "tune.cu", "general.cu", "peak.cu", "slab.cu", "persist.cu"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
           "--expt-relaxed-constexpr", "-c", os.path.join(CSRC, src), "-o", obj, *extra]
    if src.endswith(".cpp"):
        cmd = [_nvcc(), "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O3", "-x", "c++", "-c",
               os.path.join(CSRC, src), "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    if "-v" in extra and res.stderr:
        sys.stderr.write(res.stderr)
    return obj


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile and link libiffd.so; returns its path. Raises on failure."""
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = list(extra or [])
    if verbose:
        extra += ["-Xptxas", "-v"]
    with cf.ThreadPoolExecutor(max_workers=min(16, len(SOURCES))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
