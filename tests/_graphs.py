"""Small graph families with known BFS answers, and golden-fixture loading (test helpers).

Each family is built as an edge list and passed through the library's CSR builder
(``paper_1408_1605_gb300.graphs.from_edges``), the same input path every test uses."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "edges":
                pairs = [tuple(int(x) for x in tok.split("-")) for tok in rest.split()]
                out["src"] = np.array([p[0] for p in pairs], dtype=np.int32)
                out["dst"] = np.array([p[1] for p in pairs], dtype=np.int32)
            elif key == "levels":
                out["levels"] = np.array([int(x) for x in rest.split()], dtype=np.int32)
            else:
                out[key] = int(rest)
    return out


def path_edges(n):
    i = np.arange(n - 1, dtype=np.int32)
    return i, i + 1


def star_edges(n):
    leaves = np.arange(1, n, dtype=np.int32)
    return np.zeros(n - 1, dtype=np.int32), leaves


def binary_tree_edges(n):
    """Heap-indexed tree: parent of i >= 1 is (i - 1) // 2."""
    child = np.arange(1, n, dtype=np.int32)
    return (child - 1) // 2, child


def cycle_edges(n):
    i = np.arange(n, dtype=np.int32)
    return i, (i + 1) % n


def complete_edges(n):
    iu, ju = np.triu_indices(n, k=1)
    return iu.astype(np.int32), ju.astype(np.int32)


def random_edges(n, m, rng):
    return rng.integers(0, n, m).astype(np.int32), rng.integers(0, n, m).astype(np.int32)


def brute_force_distances(n, src, dst):
    """All-pairs hop distances by fixed-point relaxation d(v) <- min(d(v), d(u) + 1) over
    the undirected edge list until nothing changes (Bellman-Ford on unit weights). A
    different algorithm from a queue BFS, used to pin the oracle independently."""
    INF = n + 1
    d = np.full((n, n), INF, dtype=np.int64)
    np.fill_diagonal(d, 0)
    a = np.concatenate([src, dst]).astype(np.int64)
    b = np.concatenate([dst, src]).astype(np.int64)
    while True:
        new = d.copy()
        for col_a, col_b in zip(a, b):
            np.minimum(new[:, col_b], d[:, col_a] + 1, out=new[:, col_b])
        if np.array_equal(new, d):
            break
        d = new
    d[d >= INF] = -1
    return d.astype(np.int32)
