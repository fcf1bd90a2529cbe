"""Compile the CUDA library ``libmppi.so`` in-tree for sm_103a (GB300).

Each translation unit of ``csrc/`` is compiled by its own ``nvcc`` process in
parallel and the objects are linked into ``_build/libmppi.so``.  Rebuilds only
when a source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmppi.so")
# the bounds-checking debug build (-DMPPI_CHECKS): index checks in the rollout kernels that
# count a violation and keep the access in bounds; used by the tests, never by the planner
LIB_CHECKS = os.path.join(OUT_DIR, "libmppi_checks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
_locks = {LIB: threading.Lock(), LIB_CHECKS: threading.Lock()}   # the two builds may run side by side


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the MPPI CUDA library cannot be built")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    """Build libmppi.so, or with checks=True the bounds-checking debug build libmppi_checks.so."""
    target = LIB_CHECKS if checks else LIB
    with _locks[target]:
        if not force and not stale(target):
            return target
        os.makedirs(OUT_DIR, exist_ok=True)
        obj_dir = os.path.join(OUT_DIR, "obj_checks" if checks else "obj")
        os.makedirs(obj_dir, exist_ok=True)
        cc = nvcc()
        objs = []
        extra = ["-DMPPI_CHECKS"] if checks else []

        def compile_one(src):
            obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
            cmd = [cc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd))
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            return obj

        with ThreadPoolExecutor(max_workers=max(1, len(sources()))) as ex:
            objs = list(ex.map(compile_one, sources()))
        tmp = target + f".tmp{os.getpid()}"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, target)
        return target


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build(force=True, verbose=True, checks=True))
