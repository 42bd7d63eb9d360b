"""Named synthetic workloads (graph family, size, seeds) used by the tests and the bench.

Seeds: graph seed = GRAPH_SEED_BASE + index of the workload group below; root seed =
graph seed ^ 0x5EED. The R-MAT graphs stand in for the paper's Graph500 R-MAT inputs
(Sec. 4, Table 1: scale per GPU, edge factor 16, 64 random roots per measurement).
``edge_list_workload(path)`` wraps a graph file (e.g. one of the SNAP graphs of Table 3,
which this package does not ship) in the same interface."""
from __future__ import annotations

import fcntl
import hashlib
import os
from dataclasses import dataclass

import numpy as np

from . import graphs


@dataclass(frozen=True)
class Workload:
    name: str
    kind: str            # rmat | uniform | grid3d | edgelist
    scale: int = 0       # rmat / uniform: n = 2^scale
    edge_factor: int = 16
    dims: tuple = ()
    group: int = 0       # seed group
    roots: int = 64
    description: str = ""
    path: str = ""       # edgelist: the text edge list file

    @property
    def graph_seed(self) -> int:
        return graphs.GRAPH_SEED_BASE + self.group + (100 if self.kind == "uniform" else 0)

    @property
    def root_seed(self) -> int:
        return graphs.root_seed(self.graph_seed)

    def make(self, threads: int = 0) -> graphs.CSRGraph:
        if self.kind == "rmat":
            return graphs.rmat(self.scale, self.edge_factor, seed=self.graph_seed, threads=threads)
        if self.kind == "uniform":
            n = 1 << self.scale
            return graphs.uniform(n, self.edge_factor * n, seed=self.graph_seed, threads=threads)
        if self.kind == "grid3d":
            return graphs.grid3d(*self.dims, threads=threads)
        if self.kind == "edgelist":
            return graphs.load_edge_list(self.path, compact=True, threads=threads, name=self.name)
        raise ValueError(self.kind)

    def pick_roots(self, g: graphs.CSRGraph, k: int):
        return graphs.pick_roots(g, k, self.root_seed)

    def make_shared(self, cache_dir: str) -> graphs.CSRGraph:
        """The graph of make(), generated once per machine: the first process to take the
        lock generates it and saves offsets and columns under cache_dir; every process
        (that one included) then maps the saved arrays read-only. For runs with one process
        per GPU on one node, where every rank needs the same graph. The file names carry a
        hash of the generator source, so a changed generator does not reuse old files."""
        os.makedirs(cache_dir, exist_ok=True)
        src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "graphgen.cpp")
        with open(src, "rb") as f:
            tag = hashlib.sha256(f.read()).hexdigest()[:12]
        base = os.path.join(cache_dir, f"{self.name}-{self.graph_seed}-{tag}")
        off_path, cols_path = base + ".off.npy", base + ".cols.npy"
        with open(base + ".lock", "w") as lock:
            fcntl.flock(lock, fcntl.LOCK_EX)  # one generator; the others wait, then map the files
            try:
                if not (os.path.exists(off_path) and os.path.exists(cols_path)):
                    g = self.make()
                    for path, arr in ((off_path, g.offsets), (cols_path, g.cols)):
                        tmp = f"{path}.tmp{os.getpid()}.npy"
                        np.save(tmp, arr)
                        os.replace(tmp, path)
                    del g
            finally:
                fcntl.flock(lock, fcntl.LOCK_UN)
        off = np.load(off_path, mmap_mode="r")
        cols = np.load(cols_path, mmap_mode="r")
        return graphs.CSRGraph(len(off) - 1, off, cols, self.name)


WORKLOADS = {w.name: w for w in [
    Workload("rmat-s16-ef16", "rmat", 16, group=0, roots=16,
             description="R-MAT scale 16, edge factor 16, 16 roots (small parity case)"),
    Workload("rmat-s22-ef16", "rmat", 22, group=1, roots=64, description="R-MAT scale 22, edge factor 16, 64 roots"),
    Workload("grid3d-256", "grid3d", dims=(256, 256, 256), group=1, roots=64,
             description="3D 6-neighbour grid 256^3, non-periodic, 64 roots"),
    Workload("rmat-s26-ef16", "rmat", 26, group=2, roots=64,
             description="R-MAT scale 26, edge factor 16, 64 roots (int64 offsets in; the library narrows them to int32 when the cleaned entry count fits)"),
    Workload("uniform-s26-ef16", "uniform", 26, group=2, roots=64,
             description="uniform G(n, m), n = 2^26, m = 16 n, 64 roots"),
    Workload("rmat-s26-ef17", "rmat", 26, edge_factor=17, group=5, roots=64,
             description="R-MAT scale 26, edge factor 17: more than 2^31 - 1 CSR entries after cleaning, so the "
                         "row offsets, scan values and tile descriptors stay 64-bit"),
    Workload("rmat-s24-ef16", "rmat", 24, group=4, roots=64, description="R-MAT scale 24, edge factor 16"),
    Workload("rmat-s20-ef16", "rmat", 20, group=4, roots=64, description="R-MAT scale 20, edge factor 16"),
    Workload("grid3d-192", "grid3d", dims=(192, 192, 192), group=4, roots=64, description="3D grid 192^3"),
    Workload("uniform-n8M-deg8", "uniform", 23, edge_factor=4, group=4, roots=64,
             description="uniform G(n, m), n = 2^23, mean degree 8"),
]}


def edge_list_workload(path: str, roots: int = 64) -> Workload:
    """A graph read from a text edge list file (ids compacted to 0..n-1, every pair an
    undirected edge, loops and duplicates removed); roots are drawn like the synthetic
    workloads' from a fixed seed."""
    base = os.path.basename(path)
    for ext in (".gz", ".txt", ".tsv", ".csv", ".el", ".edges", ".mtx"):
        if base.endswith(ext):
            base = base[: -len(ext)]
    return Workload(f"edgelist-{base}", "edgelist", group=200, roots=roots, path=os.path.abspath(path),
                    description=f"edge list file {os.path.basename(path)} (ids compacted, pairs made undirected, "
                                "loops and duplicates removed)")
