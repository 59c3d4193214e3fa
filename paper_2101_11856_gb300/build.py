"""Build liblbm.so (the C-ABI CUDA library) in-tree for sm_103a with nvcc.

The library is plain CUDA C++ (no PyTorch in its interface); its translation units (SOURCES:
the step kernels of each collision model with and without free-slip faces, the immersed
boundary and diagnostics, the C ABI, the adjoint, tracers, moving solids, the radix sort and the
allocation-free force sum) are compiled in parallel and linked with the static CUDA runtime.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblbm.so")
SOURCES = ["lbm_adjoint.cu", "lbm_step_acm.cu", "lbm_step_bgk.cu", "lbm_step_raw.cu", "lbm_step_acm_fs.cu",
           "lbm_step_bgk_fs.cu", "lbm_step_raw_fs.cu", "lbm_kernels.cu", "lbm_api.cu", "lbm_tracers.cu",
           "lbm_motion.cu", "lbm_sort.cu", "lbm_static.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, "-I", CSRC] + list(extra)


def _compile(src: str, extra) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(extra)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, extra=(), verbose: bool = False) -> str:
    """Compile the library if any source is newer than it; return its path."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
        os.path.join(INCLUDE, "lbm.h")]
    if not force and os.path.exists(LIB):
        mtime = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= mtime for s in srcs):
            return LIB
    os.makedirs(BUILD, exist_ok=True)
    flags = list(extra) + (["-Xptxas", "-v"] if verbose else [])
    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, flags), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
