"""Autotuner: picks the expansion-kernel shape per (GPU, kernel kind, graph class, scale)
by timing every compiled shape on a few roots (``bfs_tune``) and remembers the choice in a
JSON cache, so later graphs of the same class and size start with the tuned shape.

Cache file: $GBFS_TUNE_CACHE, else ~/.cache/gbfs/tune.json."""
from __future__ import annotations

import json
import math
import os
import time

from . import capi


def cache_path() -> str:
    return os.environ.get("GBFS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gbfs", "tune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def key(kind: int, graph_class: str, n_vertices: int, device_name: str = "") -> str:
    if not device_name:
        try:
            import torch

            device_name = torch.cuda.get_device_name()
        except Exception:
            device_name = "gpu"
    scale = int(round(math.log2(max(n_vertices, 2))))
    kname = "single" if kind == capi.BFS_KERNEL_SINGLE else "batch"
    return f"{device_name}|{kname}|{graph_class}|s{scale}"


def lookup(k: str):
    return _load().get(k)


def apply_or_tune(graph: int, kind: int, graph_class: str, n_vertices: int, roots, levels, parents,
                  force: bool = False) -> dict:
    """Applies the cached shape for this key, or tunes and caches it. Returns the record."""
    k = key(kind, graph_class, n_vertices)
    db = _load()
    rec = db.get(k)
    count = capi.bfs_shape_count(kind)
    if rec is not None and not force and 0 <= rec.get("shape", -1) < count:
        if kind == capi.BFS_KERNEL_SINGLE and "loop" in rec:
            capi.bfs_graph_set_option(graph, capi.BFS_OPT_LOOP, rec["loop"])
            capi.bfs_graph_set_option(graph, capi.BFS_OPT_PERSIST_CTAS, rec.get("persist_ctas", 0))
        capi.bfs_graph_set_shape(graph, kind, rec["shape"])
        return dict(rec, cached=True)
    best, ms = capi.bfs_tune(graph, kind, roots, levels, parents)
    shape = best % count
    rec = {"shape": shape, "ms": ms, "shape_info": capi.bfs_shape_info(kind, shape), "when": time.time()}
    if kind == capi.BFS_KERNEL_SINGLE:
        rec["loop"] = capi.BFS_LOOP_GRAPH if best < count else capi.BFS_LOOP_PERSISTENT
        rec["persist_ctas"] = capi.bfs_graph_get_option(graph, capi.BFS_OPT_PERSIST_CTAS)
    db = _load()
    db[k] = rec
    _store(db)
    return dict(rec, cached=False)
