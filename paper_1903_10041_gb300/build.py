"""Builds the solver library ``libadmm.so`` (and, on request, the
bounds-checked ``libadmm_debug.so``) in-tree for sm_103a.

Each ``csrc/*.cu`` file is compiled separately (in parallel) with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and the
objects are linked into one shared library with the CUDA runtime linked
statically.  Objects go to ``_build/`` (``_build_dbg/``) next to this file.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
EXTRA = os.environ.get("ADMM_NVCC_FLAGS", "").split()  # extra nvcc flags (e.g. -DADMM_MIXED_VW=4)
LIB = os.path.join(HERE, "libadmm.so")
# the bounds-checked build (-DADMM_DEBUG_BOUNDS): element accesses of the mixed
# element update checked against their instance's arrays (ADMM_EBOUNDS)
DEBUG_LIB = os.path.join(HERE, "libadmm_debug.so")


def _paths(debug_bounds: bool):
    if debug_bounds:
        return os.path.join(HERE, "_build_dbg"), DEBUG_LIB
    return os.path.join(HERE, "_build"), LIB


def _flags(verbose: bool, debug_bounds: bool = False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + EXTRA
    if debug_bounds:
        f += ["-DADMM_DEBUG_BOUNDS"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(debug_bounds: bool = False) -> bool:
    lib = _paths(debug_bounds)[1]
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    bdir, lib = _paths(debug_bounds)
    if not force and up_to_date(debug_bounds):
        return lib
    os.makedirs(bdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC, *_flags(verbose, debug_bounds), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(compile_one, sources()))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug_bounds="--debug-bounds" in sys.argv))
