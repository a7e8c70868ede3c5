"""Build the CUDA library liblsh_gb300.so in-tree for sm_103a (GB300).

Each translation unit of csrc/ compiles in parallel (nvcc for .cu, g++ for
.cpp), then nvcc links the shared library next to this file.  Host code is
compiled with -ffp-contract=off (the family sampler's Box-Muller arithmetic
must be one IEEE rounding per operation).  Run: python -m paper_2503_06737_gb300.build
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblsh_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found")


def _cmds(cuda: str):
    nvcc = os.path.join(cuda, "bin", "nvcc")
    jobs = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        obj = os.path.join(OBJ, os.path.basename(src) + ".o")
        jobs.append((src, obj, [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler",
                                "-fPIC,-ffp-contract=off", "-I" + INCLUDE, "-c", src, "-o", obj]))
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cpp"))):
        obj = os.path.join(OBJ, os.path.basename(src) + ".o")
        jobs.append((src, obj, ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
                                "-I" + os.path.join(cuda, "include"), "-I" + INCLUDE, "-c", src,
                                "-o", obj]))
    return nvcc, jobs


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    cuda = _cuda_home()
    os.makedirs(OBJ, exist_ok=True)
    nvcc, jobs = _cmds(cuda)
    headers = (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
               glob.glob(os.path.join(INCLUDE, "*.h")))
    todo = [(s, o, c) for s, o, c in jobs if force or _stale(o, [s, *headers])]

    def run(job):
        src, obj, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {os.path.basename(src)}\n{' '.join(cmd)}\n{r.stdout}{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return src

    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(todo))) as ex:
            list(ex.map(run, todo))
    objs = [o for _, o, _ in jobs]
    if force or todo or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed\n{' '.join(cmd)}\n{r.stdout}{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
