"""Build the step library ``libsph_gb300.so`` in-tree for sm_103a.

Each CUDA translation unit is compiled by nvcc in parallel, then linked into
one shared library (CUDA runtime linked statically) next to this file.
Run ``python -m paper_2311_15088_gb300.build`` or call :func:`build`.
``build(checked=True)`` builds the bounds-checked variant
``libsph_gb300_checked.so`` (compiled with -DSPH_CHECK: out-of-range slot
indices of the neighbour walks set SPH_DEV_BOUNDS instead of being read);
the binding loads it when SPH_GB300_LIB names it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libsph_gb300.so")
LIB_CHECKED = os.path.join(PKG, "libsph_gb300_checked.so")

SOURCES = ["sph_api.cu", "sph_bin.cu", "sph_physics.cu", "sph_boids.cu", "sph_static.cu", "sph_mlp.cu", "sph_features.cu", "sph_surface.cu", "sph_stats.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _flags():
    return ["-O3", "-lineinfo", "-std=c++17", *ARCH, "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files + [os.path.abspath(__file__)]


def _stale(lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile and link the library if a source changed (or ``force``)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    bdir = os.path.join(BUILD_DIR, "checked") if checked else BUILD_DIR
    os.makedirs(bdir, exist_ok=True)
    flags = [*extra_flags, "-DSPH_CHECK"] if checked else list(extra_flags)
    objs = []

    def compile_one(src):
        obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
        cmd = [NVCC, "-c", os.path.join(CSRC, src), "-o", obj, *_flags(), *flags]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stdout.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [NVCC, "-shared", *ARCH, "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
