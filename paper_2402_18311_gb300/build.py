"""Compile the sm_103a placement library in-tree.

Every ``csrc/*.cu`` file is compiled to an object in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a`` and linked into
``libhybro_place.so`` next to this file (static CUDA runtime, no torch
symbols).  Objects go to ``_build/`` at the repository root.

``build(variant="bounds")`` builds the same sources with
``-DPLACE_DEBUG_BOUNDS`` into ``libhybro_place_bounds.so``: every kernel
checks the indices it forms (CSR offsets, cells, bins, tile rows) and a
failed check is returned as PLACE_EINTERNAL.  ``build_all()`` builds both.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libhybro_place.so")
BOUNDS_LIB = os.path.join(HERE, "libhybro_place_bounds.so")
VARIANTS = {"release": (LIB, OUT, []),
            "bounds": (BOUNDS_LIB, os.path.join(OUT, "bounds"), ["-DPLACE_DEBUG_BOUNDS"])}
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", ARCH,
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _compile(src, extra, out=OUT):
    obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), "-c", src, "-o", obj] + FLAGS + extra
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, extra=(), variant="release", workers=8):
    lib, out, defs = VARIANTS[variant]
    os.makedirs(out, exist_ok=True)
    srcs = sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cu"))
    with cf.ThreadPoolExecutor(max_workers=min(workers, len(srcs))) as ex:
        res = list(ex.map(lambda s: _compile(s, defs + list(extra), out), srcs))
    objs = [o for o, _ in res]
    if verbose:
        for _, err in res:
            if err:
                sys.stderr.write(err)
    tmp = lib + ".tmp"
    cmd = [nvcc(), "-shared", ARCH, "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(verbose=False):
    """Both variants, compiled side by side."""
    n = max(2, min(16, os.cpu_count() or 8))
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        fs = [ex.submit(build, verbose, (), v, n // 2) for v in VARIANTS]
        return [f.result() for f in fs]


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [],
                variant="bounds" if "--bounds" in sys.argv else "release"))
