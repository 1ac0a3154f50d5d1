"""Build the C-ABI library ``liblbm.so`` for sm_103a with nvcc (no torch).

Four translation units compile in parallel (one per storage type plus the
C ABI) and link into ``paper_1507_03521_gb300/liblbm.so``.  The FP64 unit is
built with ``--fmad=false`` so that its products and sums round separately.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "liblbm.so")
# The same sources with LBM_DEBUG defined: every population and field index
# of the single-domain kernels is bounds-checked; a failed check sets an
# error word that the next lbm_mass / lbm_laplace returns as LBM_ERR_STATE.
LIB_DEBUG = os.path.join(HERE, "liblbm_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I" + INCLUDE,
          "-I" + CSRC]
UNITS = {
    "lbm_api": [],
    "lbm_f64": ["-fmad=false"],
    "lbm_f32": [],
    "lbm_f16": [],
    "lbm_f16d": [],
    "lbm_noalloc": [],
    "lbm_batch": [],
    "lbm_slabs": [],
    "lbm3": [],
    "lbm_peaks": [],
}


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(INCLUDE, "lbm.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link liblbm.so (debug: liblbm_debug.so, with LBM_DEBUG
    defined) if any source is newer than it."""
    lib = LIB_DEBUG if debug else LIB
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    extra = ["-DLBM_DEBUG"] if debug else []
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _sources_mtime():
        return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()

    def compile_unit(name):
        obj = os.path.join(bdir, name + ".o")
        cmd = [nvcc, *ARCH, *COMMON, *extra, *UNITS[name], "-c", os.path.join(CSRC, name + ".cu"),
               "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
