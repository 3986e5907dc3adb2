"""Build libqk.so (the sm_103a CUDA library behind include/qk.h) in-tree.

Each translation unit is compiled by nvcc in parallel (one -gencode, for
sm_103a only), then linked into ``paper_2110_01792_gb300/_build/libqk.so``.
The ptxas resource report of every kernel is kept in ``_build/ptxas.log``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libqk.so")
SOURCES = ["qk_api.cu", "qk_hydro.cu", "qk_column.cu", "qk_rad.cu", "qk_rad_closures.cu",
           "qk_column_rad.cu", "qk_cell.cu", "qk_noalloc.cu", "qk_amr.cu"]
HEADERS = ["qk_internal.cuh", "qk_device.cuh", "qk_rad.cuh", "qk_ctx.cuh", "qk_exchange.cuh",
           "qk_column_rad.cuh", "qk_copy.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    paths.append(os.path.join(ROOT, "include", "qk.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def lib_path(fmad: bool = True) -> str:
    """The library of the default build, or of the diagnostic build without
    FMA contraction (``--fmad=false``: the compiler keeps every product and sum
    separately rounded; the explicit fma() calls of the sources remain)."""
    return LIB if fmad else os.path.join(BUILD + "_nofmad", "libqk.so")


def build(force: bool = False, verbose: bool = False, fmad: bool = True) -> str:
    lib = lib_path(fmad)
    bdir = os.path.dirname(lib)
    os.makedirs(bdir, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "include"), "-Xptxas", "-v"]
    if not fmad:
        flags.append("--fmad=false")

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [nvcc()] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    with open(os.path.join(bdir, "ptxas.log"), "w") as f:
        for (obj, log), src in zip(results, SOURCES):
            f.write(f"==== {src}\n{log}\n")
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}", file=sys.stderr)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
