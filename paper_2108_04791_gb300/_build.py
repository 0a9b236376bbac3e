"""Builds the CUDA library in-tree for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel and the
objects are linked into paper_2108_04791_gb300/_lib/libisprime_gb300.so.
`python -m paper_2108_04791_gb300._build [--verbose] [--debug]`.

--debug builds the same sources with IP_DEBUG_CHECKS (every queue append,
queue read and output store of the kernels bounds-checked and recorded, see
isprime_debug_checks) into _lib/libisprime_gb300_dbg.so; the package loads
it instead of the production library when ISPRIME_GB300_LIB names it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB_NAME = "libisprime_gb300.so"
LIB_PATH = os.path.join(OUT_DIR, LIB_NAME)
OBJ_DIR = os.path.join(PKG, "_build")
DEBUG_LIB_PATH = os.path.join(OUT_DIR, "libisprime_gb300_dbg.so")
DEBUG_OBJ_DIR = os.path.join(PKG, "_build_dbg")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-O2,-Wall", "-I", os.path.join(ROOT, "include")]
SOURCES = ["api.cu", "sieve.cu", "classify.cu", "mr.cu", "probe.cu", "noalloc.cu", "batched.cu",
           "autotune.cu", "server.cu", "range.cu", "small.cu", "shard.cu", "window.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "isprime.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, verbose: bool, debug: bool = False) -> tuple[str, str]:
    obj = os.path.join(DEBUG_OBJ_DIR if debug else OBJ_DIR, os.path.splitext(src)[0] + ".o")
    extra = ["-DIP_DEBUG_CHECKS"] if debug else []
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-Xptxas", "-v", "-c", os.path.join(CSRC, src),
           "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print(r.stderr, file=sys.stderr)
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compiles the library (or its debug build) if any source is newer than
    it; returns its path."""
    lib_path = DEBUG_LIB_PATH if debug else LIB_PATH
    obj_dir = DEBUG_OBJ_DIR if debug else OBJ_DIR
    if (not force and os.path.exists(lib_path)
            and os.path.getmtime(lib_path) >= _deps_mtime()):
        return lib_path
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(OUT_DIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, debug), SOURCES))
    objs = [o for o, _ in results]
    with open(os.path.join(obj_dir, "ptxas.log"), "w") as f:
        for src, (_, log) in zip(SOURCES, results):
            f.write(f"== {src}\n{log}\n")
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
                debug="--debug" in sys.argv))
