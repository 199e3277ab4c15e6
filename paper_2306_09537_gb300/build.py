"""Builds libquadswarm_gpu.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel; the objects link into one shared
library with the CUDA runtime linked statically, so the library loads on a
machine without a GPU (for the ABI tests) and on the GPU machine alike.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "_build", "libquadswarm_gpu.so")
# the debug build: the same sources with device index checks (QS_DEBUG_CHECKS)
BUILD_DEBUG = os.path.join(HERE, "_build", "debug")
LIB_DEBUG = os.path.join(HERE, "_build", "libquadswarm_gpu_debug.so")
SOURCES = ["qs_api.cu", "qs_kernels.cu", "qs_step.cu", "qs_adjoint.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libquadswarm_gpu.so")
    return path


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "qs.h"), __file__]
    return [f for f in files if os.path.isfile(f)]


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, debug: bool = False, with_debug: bool = False) -> str:
    """Builds the release library (or, debug=True, the debug build with device
    index checks); with_debug=True builds both, their translation units
    compiled in parallel. Returns the path of the (first) library."""
    variants = [True] if debug else ([False, True] if with_debug else [False])
    todo = [v for v in variants if force or not up_to_date(v)]
    if not todo:
        return LIB_DEBUG if debug else LIB
    cc = nvcc()

    def compile_one(job):
        src, dbg = job
        out_dir = BUILD_DEBUG if dbg else BUILD
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *NVCC_FLAGS, *(["-DQS_DEBUG_CHECKS"] if dbg else []), "-I" + INCLUDE, "-I" + CSRC, "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}{' (debug)' if dbg else ''}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    for dbg in todo:
        os.makedirs(BUILD_DEBUG if dbg else BUILD, exist_ok=True)
    jobs = [(src, dbg) for dbg in todo for src in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for i, dbg in enumerate(todo):
        lib = LIB_DEBUG if dbg else LIB
        tmp = lib + f".tmp{os.getpid()}"
        mine = objs[i * len(SOURCES):(i + 1) * len(SOURCES)]
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *mine, "-lcudart_static", "-lrt", "-lpthread", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB_DEBUG if debug else LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
