"""BFS oracle: TEST INFRASTRUCTURE ONLY.

A plain sequential CPU reference (``bfs_oracle.c``) for the level / predecessor arrays the
GPU library computes, plus the checks a GPU result must pass. Only ``tests/``, the smoke
check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package; the product path (``paper_1408_1605_gb300``) never does, and the two share no
code: only the seeded input generators in ``paper_1408_1605_gb300.graphs`` serve both.

Definitions followed (see ``bfs_oracle.c`` for the per-function citations):
  * level[v]: hop distance from the root, -1 if unreachable; pred[root] = root (Sec. 2.2,
    Algorithm 1; Sec. 3.2, the initialisation of Algorithm 2).
  * m_c: undirected edges inside the traversed component, the TEPS numerator (Sec. 4).
  * one top-down level (the expansion step of Algorithm 2 with R = C = 1).

Parity status: levels and m_c pinned (closed forms, brute force); parents checked by
invariants only, because ties between parents are decided by atomics (Sec. 3.4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_P64 = ctypes.POINTER(ctypes.c_int64)
_P32 = ctypes.POINTER(ctypes.c_int32)
_PU32 = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C, -O2, no vendor code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        # GBFS_ORACLE_LIB: a separately compiled oracle library, used by the test that plants
        # mistakes in copies of the oracle source to show that the pins catch them
        lib = ctypes.CDLL(os.environ.get("GBFS_ORACLE_LIB") or build())
        lib.oracle_bfs.restype = ctypes.c_int64
        lib.oracle_bfs.argtypes = [ctypes.c_int64, _P64, _P32, ctypes.c_int32, _P32, _P32]
        lib.oracle_component_edges.restype = ctypes.c_int64
        lib.oracle_component_edges.argtypes = [ctypes.c_int64, _P64, _P32]
        lib.oracle_check_tree.restype = ctypes.c_int
        lib.oracle_check_tree.argtypes = [ctypes.c_int64, _P64, _P32, ctypes.c_int32, _P32, _P32, _P32, _P64]
        lib.oracle_check_edges.restype = ctypes.c_int
        lib.oracle_check_edges.argtypes = [ctypes.c_int64, _P64, _P32, _P32, _P64]
        lib.oracle_expand_level.restype = ctypes.c_int64
        lib.oracle_expand_level.argtypes = [ctypes.c_int64, _P64, _P32, _P32, ctypes.c_int64, ctypes.c_int32,
                                            _PU32, _P32, _P32, _P32]
        _lib = lib
    return _lib


def _p(a: np.ndarray, typ):
    return a.ctypes.data_as(typ)


def _csr(offsets, cols):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    col = np.ascontiguousarray(cols, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    return off, col


def bfs(offsets, cols, root: int):
    """Sequential FIFO BFS from ``root``; returns (level int32[n], pred int32[n])."""
    off, col = _csr(offsets, cols)
    n = off.size - 1
    level = np.empty(n, dtype=np.int32)
    pred = np.empty(n, dtype=np.int32)
    r = _load().oracle_bfs(n, _p(off, _P64), _p(col, _P32), int(root), _p(level, _P32), _p(pred, _P32))
    if r < 0:
        raise ValueError("oracle_bfs: bad arguments")
    if r != int(np.count_nonzero(level >= 0)):  # the returned count is the reached set's size
        raise RuntimeError("oracle_bfs: reached count disagrees with the levels")
    return level, pred


def component_edges(offsets, level) -> int:
    """m_c = half the degree sum over reached vertices (TEPS numerator, Sec. 4)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    lv = np.ascontiguousarray(level, dtype=np.int32)
    return int(_load().oracle_component_edges(off.size - 1, _p(off, _P64), _p(lv, _P32)))


TREE_CODES = {
    0: "ok",
    1: "level differs from the oracle",
    2: "root level/pred wrong",
    3: "pred == -1 does not match level == -1",
    4: "(pred[v], v) is not a graph edge",
    5: "level[pred[v]] != level[v] - 1",
    6: "edge with |level[u] - level[v]| > 1 or reached/unreached endpoints",
}


def check_tree(offsets, cols, root: int, level_ref, level, pred):
    """Returns (code, bad_vertex); code 0 means the result is a valid BFS tree with the
    oracle's levels."""
    off, col = _csr(offsets, cols)
    ref = np.ascontiguousarray(level_ref, dtype=np.int32)
    lv = np.ascontiguousarray(level, dtype=np.int32)
    pr = np.ascontiguousarray(pred, dtype=np.int32)
    bad = ctypes.c_int64(-1)
    code = _load().oracle_check_tree(off.size - 1, _p(off, _P64), _p(col, _P32), int(root), _p(ref, _P32),
                                     _p(lv, _P32), _p(pr, _P32), ctypes.byref(bad))
    return int(code), int(bad.value)


def check_edges(offsets, cols, level):
    """Graph500-style edge check; returns (code, bad_source_vertex)."""
    off, col = _csr(offsets, cols)
    lv = np.ascontiguousarray(level, dtype=np.int32)
    bad = ctypes.c_int64(-1)
    code = _load().oracle_check_edges(off.size - 1, _p(off, _P64), _p(col, _P32), _p(lv, _P32), ctypes.byref(bad))
    return int(code), int(bad.value)


def expand_level(offsets, cols, front, lvl: int, bitmap, level, pred):
    """One top-down level in place on (bitmap, level, pred); returns the next frontier."""
    off, col = _csr(offsets, cols)
    n = off.size - 1
    fr = np.ascontiguousarray(front, dtype=np.int32)
    for a, t in ((bitmap, np.uint32), (level, np.int32), (pred, np.int32)):
        if a.dtype != t or not a.flags.c_contiguous:
            raise TypeError("bitmap/level/pred must be contiguous uint32/int32/int32 arrays")
    nxt = np.empty(max(n, 1), dtype=np.int32)
    frp = fr if fr.size else np.zeros(1, dtype=np.int32)
    c = _load().oracle_expand_level(n, _p(off, _P64), _p(col, _P32), _p(frp, _P32), fr.size, int(lvl),
                                    _p(bitmap, _PU32), _p(level, _P32), _p(pred, _P32), _p(nxt, _P32))
    return nxt[:c].copy()
