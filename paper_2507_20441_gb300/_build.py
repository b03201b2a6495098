"""Build the CUDA library for sm_103a with nvcc (in-tree, no cmake).

Each translation unit is compiled in parallel, then linked into
``_build/libtimest_gb300.so``.  Only the GB300 target is generated.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libtimest_gb300.so")
SOURCES = ["api.cu", "csr.cu", "weights.cu", "sampler.cu", "serve.cu", "tune.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the TIMEST library")
    return cand


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "timest.h"))
    return files


def build(force: bool = False, verbose: bool = False, extra_flags=None, out_dir: str = None) -> str:
    """Compile and link; `extra_flags`/`out_dir` build a variant elsewhere."""
    out_dir = out_dir or OUT_DIR
    lib = os.path.join(out_dir, "libtimest_gb300.so")
    os.makedirs(out_dir, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _inputs())
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    cc = nvcc()
    flags = FLAGS + list(extra_flags or [])
    objs = []

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{p.stderr[-4000:]}")
        if verbose and p.stderr:
            print(p.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stderr[-4000:]}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
