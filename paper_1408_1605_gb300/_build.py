"""In-tree build of the native parts: the CUDA BFS library (sm_103a) and the host graph
generator. Both are plain shared objects compiled with nvcc / g++; no cmake, no torch
extension machinery. Outputs land next to this file and are git-ignored."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

LIB_BFS = os.path.join(HERE, "libgbfs.so")
LIB_GEN = os.path.join(HERE, "libgbfs_graphgen.so")

BFS_CU = ["bfs_kernels.cu", "bfs_capi.cu", "bfs_batch_kernels.cu", "bfs_batch.cu", "bfs_serve.cu", "bfs_tune.cu", "bfs_noalloc.cu",
          "bfs_relabel.cu", "bfs_2d.cu"]


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd: list[str], verbose: bool) -> None:
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr, file=sys.stderr)


def build_graphgen(verbose: bool = False, force: bool = False) -> str:
    src = os.path.join(CSRC, "graphgen.cpp")
    if force or _stale(LIB_GEN, [src]):
        tmp = LIB_GEN + f".tmp{os.getpid()}"
        _run(["g++", "-O3", "-std=c++17", "-shared", "-fPIC", "-pthread", src, "-o", tmp], verbose)
        os.replace(tmp, LIB_GEN)
    return LIB_GEN


def _bfs_sources() -> list[str]:
    return [os.path.join(CSRC, f) for f in BFS_CU if os.path.exists(os.path.join(CSRC, f))]


def build_bfs(verbose: bool = False, force: bool = False, extra: list[str] | None = None) -> str:
    """nvcc each translation unit in parallel to an object, then link one shared library
    (static cudart, so the library loads on a machine without a GPU)."""
    srcs = _bfs_sources()
    deps = (srcs + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))
    if not (force or _stale(LIB_BFS, deps)):
        return LIB_BFS
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                    f"-I{INCLUDE}", "--expt-relaxed-constexpr"] + (extra or [])
    objs = []

    def one(src: str) -> str:
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        _run([NVCC, *flags, "-c", src, "-o", obj], verbose)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(one, srcs))
    tmp = LIB_BFS + f".tmp{os.getpid()}"
    _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"], verbose)
    os.replace(tmp, LIB_BFS)
    return LIB_BFS


def build(verbose: bool = False, force: bool = False) -> None:
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build_graphgen, verbose, force), ex.submit(build_bfs, verbose, force)]
        for f in futs:
            f.result()


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
