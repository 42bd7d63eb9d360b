"""Thin ctypes binding of the gbfs C ABI (``include/gbfs.h``): same names, argument
marshalling only. Every step of a search runs in the CUDA library; nothing here computes.

Arrays may be torch tensors (device or host) or numpy arrays (host); they are passed as raw
pointers. Streams default to torch's current CUDA stream when torch is importable.
If the shared library has not been built, every call raises ``RuntimeError``: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import _build

BFS_OK = 0
STATUS_NAMES = {
    0: "BFS_OK", 1: "BFS_ERR_INVALID_ARG", 2: "BFS_ERR_INVALID_GRAPH", 3: "BFS_ERR_OOM", 4: "BFS_ERR_CUDA",
    5: "BFS_ERR_TIMEOUT", 6: "BFS_ERR_BUSY", 7: "BFS_ERR_CANCELLED", 8: "BFS_ERR_NOT_FOUND",
}
BFS_HOST_PTRS = 0x1
BFS_DEVICE_PTRS = 0x2
BFS_OFFSETS_INT32 = 0x4
BFS_OFFSETS_INT64 = 0x8
BFS_VALIDATE = 0x10
BFS_RELABEL_DEGREE = 0x20
BFS_KEEP_INT64 = 0x40
BFS_OPT_LOOP = 1
BFS_OPT_BOTTOM_UP = 2
BFS_OPT_ALPHA = 3
BFS_OPT_BETA = 4
BFS_OPT_WAIT_LIMIT = 5
BFS_OPT_PROBE = 6
BFS_OPT_RELABELED = 7
BFS_OPT_PERSIST_CTAS = 8
BFS_OPT_WAVE_LEVELS = 9
BFS_OPT_WAVE_OVERFLOW = 10
BFS_OPT_FRONTIER = 11
BFS_OPT_UNPACKED_LEVELS = 12
BFS_OPT_WAVE_DENSE_ROWS = 13
BFS_FRONTIER_LIST = 0
BFS_FRONTIER_AUTO = 1
BFS_FRONTIER_BITMAP = 2
BFS_LOOP_PERSISTENT = 0
BFS_LOOP_GRAPH = 1
BFS_LOOP_HOST = 2
BFS_KERNEL_SINGLE = 0
BFS_KERNEL_BATCH = 1

_P = ctypes.c_void_p
_lib = None


class BfsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class bfs_serve_config(ctypes.Structure):
    _fields_ = [("memory_cap_bytes", ctypes.c_uint64), ("max_wave", ctypes.c_int32), ("queue_capacity", ctypes.c_int32),
                ("levels_per_round", ctypes.c_int32), ("waves_per_graph", ctypes.c_int32),
                ("admit_window", ctypes.c_int32), ("cohort_wait_us", ctypes.c_int32)]


class bfs_serve_report(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("levels", ctypes.c_uint64),
                ("edges_traversed", ctypes.c_int64), ("latency_p50_ms", ctypes.c_double),
                ("latency_p99_ms", ctypes.c_double), ("latency_mean_ms", ctypes.c_double),
                ("latency_max_ms", ctypes.c_double), ("wall_s", ctypes.c_double), ("gteps", ctypes.c_double),
                ("max_concurrent", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("peak_memory_bytes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class bfs_stats(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("bottom_up_levels", ctypes.c_int32), ("vertices_reached", ctypes.c_int64),
                ("edges_traversed", ctypes.c_int64), ("device_ms", ctypes.c_double), ("expand_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path() -> str:
    return _build.LIB_BFS


def declared_functions() -> list[str]:
    """Names of the functions ``include/gbfs.h`` declares."""
    with open(os.path.join(_build.INCLUDE, "gbfs.h")) as f:
        text = f.read()
    return re.findall(r"GBFS_API\s+[\w\s\*]+?\b(bfs_\w+)\s*\(", text)


def lib():
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"gbfs CUDA library not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        i64, i32, u32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        sig = {
            "bfs_graph_create": [_P, _P, i64, i64, u32, _P, ctypes.POINTER(_P)],
            "bfs_graph_destroy": [_P],
            "bfs_graph_info": [_P, ctypes.POINTER(i64), ctypes.POINTER(i64)],
            "bfs_run": [_P, i32, _P, _P, _P, ctypes.POINTER(bfs_stats)],
            "bfs_expand": [_P, _P, i64, i32, _P, _P, _P, _P, _P, _P],
            "bfs_expand_bitmap": [_P, _P, i64, i32, _P, _P, _P, _P, _P, _P, _P],
            "bfs_run_2d": [_P, ctypes.c_int, ctypes.c_int, i32, _P, _P, _P],
            "bfs_run_noalloc": [_P, _P, i64, i64, i32, _P, _P, _P],
            "bfs_run_batch": [_P, _P, ctypes.c_int, _P, _P, _P, _P],
            "bfs_serve_create": [ctypes.POINTER(bfs_serve_config), ctypes.POINTER(_P)],
            "bfs_serve_add_graph": [_P, _P, ctypes.POINTER(ctypes.c_int)],
            "bfs_serve_submit": [_P, ctypes.c_int, i32, _P, _P, ctypes.POINTER(ctypes.c_uint64)],
            "bfs_serve_poll": [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)],
            "bfs_serve_wait": [_P, ctypes.c_uint64, ctypes.c_int],
            "bfs_serve_cancel": [_P, ctypes.c_uint64],
            "bfs_serve_result": [_P, ctypes.c_uint64, ctypes.POINTER(bfs_stats)],
            "bfs_serve_stats": [_P, ctypes.POINTER(bfs_serve_report)],
            "bfs_serve_destroy": [_P],
            "bfs_shape_info": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
            "bfs_graph_set_shape": [_P, ctypes.c_int, ctypes.c_int],
            "bfs_graph_set_option": [_P, ctypes.c_int, i64],
            "bfs_level_profile": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                  ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_int)],
            "bfs_graph_get_option": [_P, ctypes.c_int, ctypes.POINTER(i64)],
            "bfs_graph_get_shape": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
            "bfs_tune": [_P, ctypes.c_int, _P, ctypes.c_int, _P, _P, _P, ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_int)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.bfs_shape_count.restype = ctypes.c_int
        L.bfs_shape_count.argtypes = [ctypes.c_int]
        L.bfs_last_error.restype = ctypes.c_char_p
        L.bfs_version.restype = ctypes.c_char_p
        _lib = L
        _extend(L)
    return _lib


_extensions = []


def _extend(L):
    for f in _extensions:
        f(L)


def check(status: int) -> None:
    if status != BFS_OK:
        raise BfsError(status, lib().bfs_last_error().decode())


def ptr(a) -> int:
    """Raw address of a torch tensor or numpy array (None -> NULL; an int passes through as
    an address). The library reads and writes flat arrays, so a strided view is refused."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("gbfs: tensor arguments must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags.c_contiguous:
            raise ValueError("gbfs: array arguments must be C-contiguous")
        return a.ctypes.data
    return int(a)


def _numel(a) -> int | None:
    if hasattr(a, "numel"):
        return int(a.numel())
    if hasattr(a, "size") and hasattr(a, "dtype"):
        return int(a.size)
    return None  # a raw address: nothing to check


def _check_int32_out(name: str, a, need: int | None = None) -> None:
    """Arrays the library writes (or reads in full) are int32 with at least `need` entries;
    checked on the host so that a wrong buffer is an exception here rather than an
    out-of-range access on the device."""
    if a is None or isinstance(a, int):
        return
    dt = str(getattr(a, "dtype", ""))
    if dt not in ("int32", "torch.int32"):
        raise ValueError(f"gbfs: {name} must be int32, got {dt or type(a).__name__}")
    k = _numel(a)
    if need is not None and k is not None and k < need:
        raise ValueError(f"gbfs: {name} holds {k} entries, the call writes {need}")


def stream_handle(stream=None) -> int:
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def bfs_graph_create(row_offsets, cols, n_vertices: int, n_entries: int, flags: int = 0, stream=None) -> int:
    out = _P()
    check(lib().bfs_graph_create(ptr(row_offsets), ptr(cols), int(n_vertices), int(n_entries), int(flags),
                                 stream_handle(stream), ctypes.byref(out)))
    return out.value


def bfs_graph_destroy(graph: int) -> None:
    check(lib().bfs_graph_destroy(graph))


def bfs_graph_info(graph: int) -> tuple[int, int]:
    n, m = ctypes.c_int64(), ctypes.c_int64()
    check(lib().bfs_graph_info(graph, ctypes.byref(n), ctypes.byref(m)))
    return n.value, m.value


def bfs_run(graph: int, root: int, levels, parents, stream=None, want_stats: bool = False):
    _check_int32_out("levels", levels)
    _check_int32_out("parents", parents)
    if _numel(levels) is not None or _numel(parents) is not None:
        n = bfs_graph_info(graph)[0]
        _check_int32_out("levels", levels, n)
        _check_int32_out("parents", parents, n)
    st = bfs_stats()
    check(lib().bfs_run(graph, int(root), ptr(levels), ptr(parents), stream_handle(stream),
                        ctypes.byref(st) if want_stats else None))
    return st if want_stats else None


def bfs_run_batch(graph: int, roots, levels, parents, stream=None, want_stats: bool = False):
    """roots: host int32 array (<= 64); levels / parents: int32[len(roots)][n]."""
    import numpy as np

    r = np.ascontiguousarray(roots, dtype=np.int32)
    _check_int32_out("levels", levels)
    _check_int32_out("parents", parents)
    if 1 <= r.size <= 64 and (_numel(levels) is not None or _numel(parents) is not None):
        need = r.size * bfs_graph_info(graph)[0]
        _check_int32_out("levels", levels, need)
        _check_int32_out("parents", parents, need)
    st = (bfs_stats * max(1, r.size))()
    check(lib().bfs_run_batch(graph, r.ctypes.data, int(r.size), ptr(levels), ptr(parents), stream_handle(stream),
                              st if want_stats else None))
    return list(st)[: r.size] if want_stats else None


def bfs_expand(graph: int, frontier, n_frontier: int, level: int, bitmap, levels, parents, next_, next_count,
               stream=None) -> None:
    check(lib().bfs_expand(graph, ptr(frontier), int(n_frontier), int(level), ptr(bitmap), ptr(levels), ptr(parents),
                           ptr(next_), ptr(next_count), stream_handle(stream)))


def bfs_run_2d(graph: int, R: int, C: int, root: int, levels, parents, stream=None) -> None:
    if _numel(levels) is not None or _numel(parents) is not None:
        n = bfs_graph_info(graph)[0]
        _check_int32_out("levels", levels, n)
        _check_int32_out("parents", parents, n)
    check(lib().bfs_run_2d(graph, int(R), int(C), int(root), ptr(levels), ptr(parents), stream_handle(stream)))


def bfs_expand_bitmap(graph: int, frontier, n_frontier: int, level: int, bitmap, levels, parents, next_bitmap,
                      next_, next_count, stream=None) -> None:
    check(lib().bfs_expand_bitmap(graph, ptr(frontier), int(n_frontier), int(level), ptr(bitmap), ptr(levels),
                                  ptr(parents), ptr(next_bitmap), ptr(next_), ptr(next_count), stream_handle(stream)))


def bfs_run_noalloc(row_offsets, cols, n_vertices: int, n_entries: int, root: int, levels, parents,
                    stream=None) -> None:
    # every array is read or written in full on the device: check types and sizes here
    _check_int32_out("row_offsets", row_offsets, int(n_vertices) + 1)
    if int(n_entries) > 0:
        _check_int32_out("cols", cols, int(n_entries))
    _check_int32_out("levels", levels, int(n_vertices))
    _check_int32_out("parents", parents, int(n_vertices))
    check(lib().bfs_run_noalloc(ptr(row_offsets), ptr(cols), int(n_vertices), int(n_entries), int(root),
                                ptr(levels), ptr(parents), stream_handle(stream)))


def bfs_serve_create(memory_cap_bytes: int = 0, max_wave: int = 0, queue_capacity: int = 0,
                     levels_per_round: int = 0, waves_per_graph: int = 0, admit_window: int = 0,
                     cohort_wait_us: int = 0) -> int:
    cfg = bfs_serve_config(int(memory_cap_bytes), int(max_wave), int(queue_capacity), int(levels_per_round),
                           int(waves_per_graph), int(admit_window), int(cohort_wait_us))
    out = _P()
    check(lib().bfs_serve_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def bfs_serve_add_graph(server: int, graph: int) -> int:
    gid = ctypes.c_int()
    check(lib().bfs_serve_add_graph(server, graph, ctypes.byref(gid)))
    return gid.value


def bfs_serve_submit(server: int, graph_id: int, root: int, levels, parents) -> int:
    _check_int32_out("levels", levels)
    _check_int32_out("parents", parents)
    t = ctypes.c_uint64()
    check(lib().bfs_serve_submit(server, int(graph_id), int(root), ptr(levels), ptr(parents), ctypes.byref(t)))
    return t.value


def bfs_serve_poll(server: int, ticket: int) -> bool:
    d = ctypes.c_int()
    check(lib().bfs_serve_poll(server, int(ticket), ctypes.byref(d)))
    return bool(d.value)


def bfs_serve_wait(server: int, ticket: int, timeout_ms: int = 60000) -> None:
    check(lib().bfs_serve_wait(server, int(ticket), int(timeout_ms)))


def bfs_serve_cancel(server: int, ticket: int) -> None:
    check(lib().bfs_serve_cancel(server, int(ticket)))


def bfs_serve_result(server: int, ticket: int) -> bfs_stats:
    st = bfs_stats()
    check(lib().bfs_serve_result(server, int(ticket), ctypes.byref(st)))
    return st


def bfs_serve_stats(server: int) -> dict:
    rep = bfs_serve_report()
    check(lib().bfs_serve_stats(server, ctypes.byref(rep)))
    return rep.as_dict()


def bfs_serve_destroy(server: int) -> None:
    check(lib().bfs_serve_destroy(server))


def bfs_graph_set_option(graph: int, option: int, value: int) -> None:
    check(lib().bfs_graph_set_option(graph, int(option), int(value)))


def bfs_graph_get_option(graph: int, option: int) -> int:
    v = ctypes.c_int64()
    check(lib().bfs_graph_get_option(graph, int(option), ctypes.byref(v)))
    return v.value


def bfs_level_profile(graph: int, cap: int = 64) -> list[dict]:
    ms = (ctypes.c_double * cap)()
    nf = (ctypes.c_int64 * cap)()
    bu = (ctypes.c_int32 * cap)()
    n = ctypes.c_int()
    check(lib().bfs_level_profile(graph, int(cap), ms, nf, bu, ctypes.byref(n)))
    return [{"ms": ms[i], "frontier": nf[i], "bottom_up": bool(bu[i])} for i in range(min(n.value, cap))]


def bfs_shape_count(kind: int) -> int:
    return int(lib().bfs_shape_count(int(kind)))


def bfs_shape_info(kind: int, shape: int) -> dict:
    b, e, c, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().bfs_shape_info(int(kind), int(shape), ctypes.byref(b), ctypes.byref(e), ctypes.byref(c),
                               ctypes.byref(w)))
    return {"block": b.value, "edges_per_thread": e.value, "claim_buffer": c.value, "warp_tiles": w.value}


def bfs_graph_set_shape(graph: int, kind: int, shape: int) -> None:
    check(lib().bfs_graph_set_shape(graph, int(kind), int(shape)))


def bfs_graph_get_shape(graph: int, kind: int) -> int:
    s = ctypes.c_int()
    check(lib().bfs_graph_get_shape(graph, int(kind), ctypes.byref(s)))
    return s.value


def bfs_tune(graph: int, kind: int, roots, levels, parents, stream=None):
    """Returns (best candidate, [ms per candidate]); single-source candidates are
    (graph loop, shape 0..count-1), (persistent loop, shape 0..count-1), then (persistent
    loop with 2 CTAs per SM, shape 0..count-1), then (with 1 CTA per SM, shape 0..count-1)."""
    import numpy as np

    r = np.ascontiguousarray(roots, dtype=np.int32)
    _check_int32_out("levels", levels)
    _check_int32_out("parents", parents)
    single = kind == BFS_KERNEL_SINGLE
    if (single or 1 <= r.size <= 64) and (_numel(levels) is not None or _numel(parents) is not None):
        need = bfs_graph_info(graph)[0] * (1 if single else r.size)
        _check_int32_out("levels", levels, need)
        _check_int32_out("parents", parents, need)
    n = bfs_shape_count(kind) * (4 if kind == BFS_KERNEL_SINGLE else 1)
    ms = (ctypes.c_double * max(n, 1))()
    best = ctypes.c_int(-1)
    check(lib().bfs_tune(graph, int(kind), r.ctypes.data, int(r.size), ptr(levels), ptr(parents),
                         stream_handle(stream), ms, ctypes.byref(best)))
    return best.value, [ms[i] for i in range(n)]


def bfs_last_error() -> str:
    return lib().bfs_last_error().decode()


def bfs_version() -> str:
    return lib().bfs_version().decode()
