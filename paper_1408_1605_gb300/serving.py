"""Seeded Poisson load driver for the serving C ABI (``bfs_serve_*``).

Only request generation and bookkeeping live here: arrival times are exponential gaps at
``rate`` queries/s from a seeded generator, roots are uniform over each graph's vertices,
and every query goes to the server through ``bfs_serve_submit``. The searches themselves
run in the CUDA library."""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import capi


@dataclass
class Query:
    graph_id: int
    root: int
    levels: object
    parents: object
    ticket: int = 0
    t_submit: float = 0.0


@dataclass
class LoadResult:
    queries: list = field(default_factory=list)
    busy_retries: int = 0
    offered_s: float = 0.0


def poisson_schedule(n_queries: int, rate: float, n_vertices: list[int], seed: int):
    """(arrival offset s, graph index, root) for each query; graph chosen uniformly."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_queries)
    arrivals = np.cumsum(gaps) - gaps[0]
    gsel = rng.integers(0, len(n_vertices), n_queries)
    roots = np.array([rng.integers(0, n_vertices[g]) for g in gsel], dtype=np.int64)
    return arrivals, gsel, roots


def run_poisson(server: int, graph_ids: list[int], n_vertices: list[int], n_queries: int, rate: float, seed: int,
                alloc, timeout_s: float = 300.0) -> LoadResult:
    """Submits n_queries at Poisson arrivals, then waits for all. ``alloc(n)`` returns a
    (levels, parents) pair of int32[n] buffers (device tensors or host arrays)."""
    arrivals, gsel, roots = poisson_schedule(n_queries, rate, n_vertices, seed)
    out = LoadResult()
    t0 = time.perf_counter()
    for i in range(n_queries):
        target = t0 + arrivals[i]
        while True:
            now = time.perf_counter()
            if now >= target:
                break
            time.sleep(min(target - now, 0.0005))
        g = int(gsel[i])
        lv, pr = alloc(n_vertices[g])
        q = Query(graph_ids[g], int(roots[i]), lv, pr)
        while True:
            try:
                q.ticket = capi.bfs_serve_submit(server, q.graph_id, q.root, lv, pr)
                break
            except capi.BfsError as e:
                if e.status != 6:  # BFS_ERR_BUSY
                    raise
                out.busy_retries += 1
                time.sleep(0.0005)
        q.t_submit = time.perf_counter()
        out.queries.append(q)
    out.offered_s = time.perf_counter() - t0
    deadline = time.perf_counter() + timeout_s
    for q in out.queries:
        capi.bfs_serve_wait(server, q.ticket, max(1, int(1000 * (deadline - time.perf_counter()))))
    return out
