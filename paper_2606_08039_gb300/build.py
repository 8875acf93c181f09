"""Builds the CUDA library libmdg.so in-tree for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel to an object file, then the
objects are linked into paper_2606_08039_gb300/_lib/libmdg.so (static CUDA runtime, so
the library loads on machines without a GPU driver; the first CUDA call then fails).
Run `python -m paper_2606_08039_gb300.build` or call build_library().
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB_NAME = "libmdg.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmdg.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INCLUDE, "mdg.h"), __file__]


DEBUG_LIB_NAME = "libmdg_debug.so"


def lib_path(debug: bool = False) -> str:
    return os.path.join(OUT_DIR, DEBUG_LIB_NAME if debug else LIB_NAME)


def up_to_date(debug: bool = False) -> bool:
    p = lib_path(debug)
    if not os.path.exists(p):
        return False
    t = os.path.getmtime(p)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build_library(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a and link libmdg.so (debug=True: libmdg_debug.so with
    -DMDG_DEBUG, whose kernels check their table indices and report MDG_STATUS_BOUNDS).
    Returns the library path."""
    if not force and up_to_date(debug):
        return lib_path(debug)
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                     "--expt-relaxed-constexpr"]
    if ptxas_info:
        common += ["-Xptxas", "-v"]
    if debug:
        common += ["-DMDG_DEBUG"]

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src) + f".{'d' if debug else 'r'}{os.getpid()}.o")
        cmd = [nvcc, *common, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(_sources()))) as ex:
        results = list(ex.map(compile_one, _sources()))
    if verbose or ptxas_info:
        for _, log in results:
            if log.strip():
                print(log, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = lib_path(debug) + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path(debug))
    return lib_path(debug)


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True, ptxas_info="-v" in sys.argv))
