"""Builds libtosolve.so (the C ABI of include/tosolve.h) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then
linked into one shared library next to this file.  No cmake; a rebuild is
skipped when the library is newer than every source.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libtosolve.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["k_setup.cu", "k_solve.cu", "k_grad.cu", "k_tc.cu", "k_tc2.cu", "k_noalloc.cu", "k_q2.cu", "k_fix.cu", "k_thresh.cu", "tosolve_api.cu", "tosolve_server.cpp", "pool.cpp", "tune.cpp"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtosolve.so")


def _sources():
    srcs = [os.path.join(CSRC, u) for u in UNITS]
    deps = srcs + [os.path.join(CSRC, "internal.cuh"), os.path.join(CSRC, "dfloat.cuh"),
                   os.path.join(CSRC, "pool.h"),
                   os.path.join(os.path.dirname(HERE), "include", "tosolve.h")]
    return srcs, deps


def build(force: bool = False, verbose: bool = False) -> str:
    srcs, deps = _sources()
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "--expt-relaxed-constexpr", "-Xptxas", "-v" if verbose else "-O3"]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for _, err in results:
            sys.stderr.write(err)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-Xlinker", "--no-undefined", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
