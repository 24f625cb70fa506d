"""Builds libwq.so (the C-ABI library) in-tree for sm_103a.

Usage: python -m paper_1710_01048_gb300.build [--force] [--verbose]

Each translation unit compiles in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a); host code is compiled without FMA
contraction so the host rule tables are identical on x86_64 and aarch64, and
device code contracts nothing the source does not write as an FMA.
Outputs go to paper_1710_01048_gb300/_build/ (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libwq.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# --fmad=false: device code gets a fused multiply-add only where the source
# asks for one (fma/fmaf); the double-float arithmetic's error-free
# transformations need every other product and sum rounded on its own, and
# every kernel instantiation then computes the same bits.
CU_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC", "-Xcompiler",
                   "-ffp-contract=off", "--expt-relaxed-constexpr", "-I", INCLUDE]
CXX_FLAGS = ["-O2", "-fPIC", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-I", INCLUDE,
             "-I", os.path.join(CUDA_HOME, "include")]

SOURCES = ["rules.cpp", "api.cu", "rows_p2_double.cu", "rows_p3_double.cu", "rows_p2_float.cu", "rows_p3_float.cu",
           "rows_p2_dd.cu", "rows_p3_dd.cu", "noalloc.cu", "batch.cu", "batch_double.cu", "batch_float.cu",
           "batch_dd.cu", "csr.cu", "general.cu", "tune_cache.cpp"]
HEADERS = ["wq_internal.h", "checked.cuh", "assemble.cuh", "launch.cuh", "dd.cuh", "adjoint.cuh", "fold.cuh", "batch.cuh", "ukernel.cuh"]


def _newest_dep():
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "wq.h"), os.path.abspath(__file__)]
    return max(os.path.getmtime(d) for d in deps)


def _compile(src, force, verbose, out, extra):
    path = os.path.join(CSRC, src)
    obj = os.path.join(out, src.replace(".", "_") + ".o")
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(path), _newest_dep()):
        return obj
    if src.endswith(".cu"):
        cmd = [NVCC] + CU_FLAGS + list(extra) + ["-c", path, "-o", obj + ".tmp"]
    else:
        cmd = ["g++"] + CXX_FLAGS + ["-c", path, "-o", obj + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {src}\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr.strip():
        print(r.stderr, file=sys.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, out_dir: str = OUT, extra_nvcc=()) -> str:
    """Compiles and links libwq.so into out_dir (default: the in-tree _build);
    returns its path.  Incremental unless force.  extra_nvcc: additional nvcc
    flags (e.g. -D tuning macros) for the CUDA sources."""
    if shutil.which(NVCC) is None and not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libwq.so")
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, verbose, out_dir, extra_nvcc), SOURCES))
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        lib64 = os.path.join(CUDA_HOME, "lib64")
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + ["-Xlinker", f"-rpath,{lib64}"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB)
