"""Builds libpc.so (all CUDA sources under csrc/) in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into ``_build/libpc.so``.  The same sources compiled with
-DPC_MAX_D=10 link into ``_build/libpc_d10.so``, the build for input
dimensions 9 and 10 (libpc.so takes D <= 8).  Rebuilds only when a source or
header is newer than a library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpc.so")
LIB_D10 = os.path.join(BUILD, "libpc_d10.so")
VARIANTS = {LIB: [], LIB_D10: ["-DPC_MAX_D=10"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale() -> bool:
    if not all(os.path.exists(lib) for lib in VARIANTS):
        return True
    t = min(os.path.getmtime(lib) for lib in VARIANTS)
    return any(os.path.getmtime(p) > t for p in _deps())


def _objdir(lib: str) -> str:
    return BUILD if lib == LIB else os.path.join(BUILD, os.path.basename(lib)[:-3])


def _compile(src: str, lib: str, verbose: bool) -> str:
    os.makedirs(_objdir(lib), exist_ok=True)
    obj = os.path.join(_objdir(lib), os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC] + ARCH + FLAGS + VARIANTS[lib] + ["-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and not _stale():
        return LIB
    srcs = _sources()
    jobs = [(src, lib) for lib in VARIANTS for src in srcs]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda j: _compile(j[0], j[1], verbose), jobs))
    for lib in VARIANTS:
        tmp = lib + f".tmp{os.getpid()}"
        mine = [o for o, (_, l) in zip(objs, jobs) if l == lib]
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + mine + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
