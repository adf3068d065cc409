"""Build libdot.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

Each .cu file under csrc/ is compiled by nvcc in parallel into _build/, then
linked into paper_2604_21566_gb300/libdot.so with the CUDA runtime linked
statically.  The microbenchmarks under csrc/probe/ (the peaks the bench
reports kernels against; no arithmetic of the library) are linked into
libdotprobe.so the same way.  Rebuilds only what changed.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdot.so")
PROBE_LIB = os.path.join(PKG, "libdotprobe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: libdot needs the CUDA toolkit to build")
    return p


def _sources(sub: str = ""):
    return sorted(glob.glob(os.path.join(CSRC, sub, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra_flags=None, jobs: int | None = None) -> str:
    """Build libdot.so and libdotprobe.so; returns the path of libdot.so."""
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    hdrs = _headers()
    flags = FLAGS + list(extra_flags or [])
    libs = ((LIB, _sources(), ""), (PROBE_LIB, _sources("probe"), "probe_"))
    todo = []
    objs = {}
    for lib, srcs, prefix in libs:
        objs[lib] = []
        for src in srcs:
            obj = os.path.join(BUILD, prefix + os.path.basename(src)[:-3] + ".o")
            objs[lib].append(obj)
            if _stale(obj, [src] + hdrs):
                todo.append((src, obj))

    def compile_one(job):
        src, obj = job
        cmd = [nv, *ARCH, *flags, "-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return r.stderr

    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 4)
        with ThreadPoolExecutor(max_workers=n) as ex:
            for msg in ex.map(compile_one, todo):
                if verbose and msg:
                    print(msg)
    for lib, _, _ in libs:
        if todo or _stale(lib, objs[lib]):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs[lib]]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stderr}")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
