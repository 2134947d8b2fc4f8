"""Builds the CUDA library ``libmdgb300.so`` in-tree with nvcc for sm_103a.

Each ``csrc/*.cu`` is compiled in parallel to ``_build/*.o`` and linked into
``paper_2009_07400_gb300/libmdgb300.so`` against the shared CUDA runtime (so a
process that already loaded PyTorch's runtime shares it).  No CMake.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmdgb300.so")
# the bounds-checked variant (MD_DEBUG_CHECKS=1): every gathered or stored
# index is checked on the device and a bad one raises an error flag
DEBUG_OUT_DIR = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(HERE, "libmdgb300_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-diag-suppress", "1444"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False,
          cell_tile: int = 2) -> str:
    """Compiles (if needed) and returns the path of libmdgb300.so, or with
    debug=True of the bounds-checked libmdgb300_debug.so.  cell_tile (1, 2
    or 4): the edge of the cell tiles that number the cells (and so order the
    atoms); the library uses 2, and the others build libmdgb300_tile1.so /
    libmdgb300_tile4.so for the cell-order study of bench.py."""
    if cell_tile not in (1, 2, 4) or (debug and cell_tile != 2):
        raise ValueError("cell_tile must be 1, 2 or 4 (2 for the debug build)")
    nvcc = _nvcc()
    out_dir, lib = (DEBUG_OUT_DIR, DEBUG_LIB) if debug else (OUT_DIR, LIB)
    if cell_tile != 2:
        out_dir = os.path.join(HERE, f"_build_tile{cell_tile}")
        lib = os.path.join(HERE, f"libmdgb300_tile{cell_tile}.so")
    flags = NVCC_FLAGS + (["-DMD_DEBUG_CHECKS=1"] if debug else []) + (
        [f"-DMD_CELL_TILE={cell_tile}"] if cell_tile != 2 else [])
    os.makedirs(out_dir, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(os.path.dirname(HERE), "include", "*.h"))
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append((src, obj))

    def compile_one(job):
        src, obj = job
        cmd = [nvcc] + ARCH + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr)
        return obj

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(compile_one, jobs))
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        libdir = _cuda_lib_dir(nvcc)
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
            "-Xlinker", f"-rpath,{libdir}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
