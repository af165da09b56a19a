"""In-tree build of the CUDA library libmbs.so for sm_103a (GB300).

Each translation unit (CUDA, and the host-only ``.cpp``) is compiled by nvcc in
parallel into ``_build/`` and the objects are linked into ``libmbs.so`` next to
this file.  A rebuild happens
only when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmbs.so")
SOURCES = ["capi.cu", "gmatvec.cu", "gumma.cu", "blas.cu", "sbuild.cu", "peaks.cu", "serve.cu",
           "noalloc.cu", "gdf.cu", "blsq.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "-diag-suppress", "177"]
# single-precision G_hat kernels: flush denormals, approximate division / square
# root (these flags touch FP32 arithmetic only; the FP64 kernels are unaffected)
EXTRA = {f: ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"] for f in ("gmatvec.cu", "gumma.cu")}
# double-float kernel: no contraction of a separate multiply and add into a
# fused multiply-add, which would break the exact error terms of the two-sum
# and two-product transformations (explicit fmaf / fma calls stay fused)
EXTRA["gdf.cu"] = ["-fmad=false"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmbs.so")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h", ".cpp"))]
    files.append(os.path.join(INCLUDE, "mbs.h"))
    return files


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *EXTRA.get(src, []), "-I", INCLUDE, "-c",
               os.path.join(CSRC, src), "-o", obj]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{p.stderr}")
        if verbose and p.stderr:
            print(p.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread",
           "-Xlinker", "-rpath", "-Xlinker", cuda_lib]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
