"""Build the CUDA library in-tree: one sm_103a shared object.

Compiles every ``csrc/*.cu`` translation unit with nvcc in parallel
(``-gencode arch=compute_103a,code=sm_103a``, ``-lineinfo``) and links them
into ``_lib/liblm_gb300.so`` with the CUDA runtime linked statically, so the
library loads next to PyTorch's own runtime.  Rebuilds only what changed.

``build(debug_bounds=True)`` builds the bounds-checked variant
``_lib/liblm_gb300_debug.so`` (``-DLM_DEBUG_BOUNDS``: device index checks that
record the first out-of-range access and skip it; ``lm_debug_check`` reports
them).  The Python binding loads it when ``LM_DEBUG_BOUNDS=1`` is set.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIB = os.path.join(LIBDIR, "liblm_gb300.so")
OBJDIR_DEBUG = os.path.join(LIBDIR, "obj_debug")
LIB_DEBUG = os.path.join(LIBDIR, "liblm_gb300_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
              "-Wno-deprecated-gpu-targets"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build the library")


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def build(verbose: bool = False, force: bool = False, debug_bounds: bool = False) -> str:
    nvcc = _nvcc()
    objdir = OBJDIR_DEBUG if debug_bounds else OBJDIR
    lib = LIB_DEBUG if debug_bounds else LIB
    extra = ["-DLM_DEBUG_BOUNDS"] if debug_bounds else []
    os.makedirs(objdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_t = _headers_mtime()
    jobs = []
    objs = []
    for src in srcs:
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_t):
            jobs.append([nvcc, *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if jobs or not os.path.exists(lib) or force:
        tmp = lib + ".tmp%d" % os.getpid()
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
