"""Build the CUDA library ``_build/libata.so`` in-tree (sm_103a only).

Every translation unit is compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a -lineinfo``) and linked into one
shared library exporting the C ABI of ``include/ata.h``.  Nothing here imports
torch; the library has no torch types in its interface.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libata.so")

CUDA_UNITS = ["ata_api.cu", "kernels.cu", "leaf_tc.cu", "noalloc.cu"]
CXX_UNITS = ["plan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _stale(objs) -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    srcs.append(os.path.join(ROOT, "include", "ata.h"))
    srcs.append(os.path.abspath(__file__))
    return any(os.path.getmtime(s) > t for s in srcs if os.path.exists(s))


def build(verbose: bool = False, force: bool = False, ptxas_verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and not _stale(None):
        return LIB
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", SRC]
    cu_flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                       "--expt-relaxed-constexpr", "-Xcompiler", "-fno-strict-aliasing"] + inc
    if ptxas_verbose:
        cu_flags += ["-Xptxas", "-v"]
    jobs = []
    for u in CUDA_UNITS:
        obj = os.path.join(OUT, u + ".o")
        jobs.append([nvcc] + cu_flags + ["-c", os.path.join(SRC, u), "-o", obj])
    for u in CXX_UNITS:
        obj = os.path.join(OUT, u + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall"] + inc +
                    ["-c", os.path.join(SRC, u), "-o", obj])
    logs = []
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for out in ex.map(_run, jobs):
            logs.append(out)
    objs = [os.path.join(OUT, u + ".o") for u in CUDA_UNITS + CXX_UNITS]
    tmp = LIB + ".tmp"
    logs.append(_run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs))
    os.replace(tmp, LIB)
    if verbose or ptxas_verbose:
        print("\n".join(l for l in logs if l.strip()))
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv)
    print(LIB)
