"""Seeded synthetic graph inputs and the symmetric CSR builder (host side).

Input preparation only: shared by the CPU oracle tests and the GPU path, and holding none
of the BFS arithmetic. The heavy lifting is in ``csrc/graphgen.cpp`` (multithreaded,
counter-based randomness, so the result does not depend on the thread count).

Workloads (stand-ins for the paper's Graph500 R-MAT inputs, Sec. 4; the Graph500 generator
itself is not available, so byte parity with it is not claimed):
  * ``rmat(scale, edge_factor)``: edge_factor * 2^scale generated pairs, quadrant
    probabilities A/B/C/D = .57/.19/.19/.05, seeded vertex permutation, self-loops and
    duplicates removed, symmetrized.
  * ``uniform(n, m)``: G(n, m) pairs with both endpoints uniform, same cleaning.
  * ``grid3d(X, Y, Z)``: non-periodic 6-neighbour grid, id = x + X * (y + Y * z).

Graphs from files: ``load_edge_list(path)`` reads a text edge list (one "u v" pair per line,
the form in which SNAP distributes the real-world graphs of the paper's Table 3, Sec. 5) or a
MatrixMarket coordinate file, optionally gzip-compressed, and builds the same cleaned
symmetric CSR.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

_lib = None
_P64 = ctypes.POINTER(ctypes.c_int64)
_P32 = ctypes.POINTER(ctypes.c_int32)

# Seeds: graph seed = GRAPH_SEED_BASE + workload index; root seed = graph seed ^ 0x5EED.
GRAPH_SEED_BASE = 20140806


def _load():
    global _lib
    if _lib is None:
        path = _build.LIB_GEN
        if not os.path.exists(path):
            _build.build_graphgen()
        lib = ctypes.CDLL(path)
        lib.gg_rmat_edges.restype = ctypes.c_int
        lib.gg_rmat_edges.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.c_int, _P32, _P32, ctypes.c_int]
        lib.gg_uniform_edges.restype = ctypes.c_int
        lib.gg_uniform_edges.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, _P32, _P32, ctypes.c_int]
        lib.gg_grid3d_edge_count.restype = ctypes.c_int64
        lib.gg_grid3d_edge_count.argtypes = [ctypes.c_int64] * 3
        lib.gg_grid3d_edges.restype = ctypes.c_int
        lib.gg_grid3d_edges.argtypes = [ctypes.c_int64] * 3 + [_P32, _P32, ctypes.c_int]
        lib.gg_build_csr.restype = ctypes.c_int64
        lib.gg_build_csr.argtypes = [ctypes.c_int64, ctypes.c_int64, _P32, _P32, _P64, _P32, ctypes.c_int]
        lib.gg_parse_edge_list.restype = ctypes.c_int64
        lib.gg_parse_edge_list.argtypes = [ctypes.c_void_p, ctypes.c_int64, _P32, _P32, ctypes.c_int64, _P64, _P64,
                                           ctypes.c_int]
        lib.gg_pick_roots.restype = ctypes.c_int64
        lib.gg_pick_roots.argtypes = [ctypes.c_int64, _P64, ctypes.c_int64, ctypes.c_uint64, _P32]
        _lib = lib
    return _lib


@dataclass
class CSRGraph:
    """Symmetric CSR: ``offsets`` int64[n + 1], ``cols`` int32[nnz], rows sorted. ``ids``:
    for a graph loaded with its ids compacted, the file id of each vertex (else None)."""

    n: int
    offsets: np.ndarray
    cols: np.ndarray
    name: str = ""
    ids: np.ndarray | None = None

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)

    def offsets32(self) -> np.ndarray:
        if self.nnz > np.iinfo(np.int32).max:
            raise OverflowError("graph has more than 2^31 - 1 CSR entries; int64 offsets needed")
        return self.offsets.astype(np.int32)


def _p(a, typ):
    return a.ctypes.data_as(typ)


def rmat_edges(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               seed: int = GRAPH_SEED_BASE, permute: bool = True, threads: int = 0):
    m = int(edge_factor) << int(scale)
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    r = _load().gg_rmat_edges(int(scale), m, a, b, c, int(seed) & (2**64 - 1), int(bool(permute)),
                              _p(src, _P32), _p(dst, _P32), int(threads))
    if r != 0:
        raise ValueError("gg_rmat_edges: bad arguments")
    return src, dst


def uniform_edges(n: int, m: int, seed: int, threads: int = 0):
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    if _load().gg_uniform_edges(int(n), int(m), int(seed) & (2**64 - 1), _p(src, _P32), _p(dst, _P32),
                                int(threads)) != 0:
        raise ValueError("gg_uniform_edges: bad arguments")
    return src, dst


def grid3d_edges(X: int, Y: int, Z: int, threads: int = 0):
    m = int(_load().gg_grid3d_edge_count(X, Y, Z))
    if m < 0:
        raise ValueError("grid dimensions must be >= 1")
    src = np.empty(max(m, 1), dtype=np.int32)
    dst = np.empty(max(m, 1), dtype=np.int32)
    if _load().gg_grid3d_edges(X, Y, Z, _p(src, _P32), _p(dst, _P32), int(threads)) != 0:
        raise ValueError("gg_grid3d_edges: bad arguments")
    return src[:m], dst[:m]


def from_edges(n: int, src, dst, threads: int = 0, name: str = "") -> CSRGraph:
    """Symmetric, loop-free, duplicate-free CSR with sorted rows from an edge list."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    if src.shape != dst.shape:
        raise ValueError("src/dst length mismatch")
    m = src.size
    offsets = np.empty(n + 1, dtype=np.int64)
    cols = np.empty(max(2 * m, 1), dtype=np.int32)
    sp = src if m else np.zeros(1, dtype=np.int32)
    dp = dst if m else np.zeros(1, dtype=np.int32)
    nnz = _load().gg_build_csr(int(n), m, _p(sp, _P32), _p(dp, _P32), _p(offsets, _P64), _p(cols, _P32),
                               int(threads))
    if nnz == -3:
        raise ValueError("edge endpoint out of range")
    if nnz < 0:
        raise MemoryError("gg_build_csr failed") if nnz == -2 else ValueError("gg_build_csr: bad arguments")
    if nnz < cols.size // 2:
        cols = cols[:nnz].copy()
    else:
        cols = cols[:nnz]
    return CSRGraph(int(n), offsets, cols, name)


def rmat(scale: int, edge_factor: int = 16, seed: int = GRAPH_SEED_BASE, threads: int = 0, **kw) -> CSRGraph:
    src, dst = rmat_edges(scale, edge_factor, seed=seed, threads=threads, **kw)
    g = from_edges(1 << scale, src, dst, threads=threads, name=f"rmat-s{scale}-ef{edge_factor}")
    return g


def uniform(n: int, m: int, seed: int, threads: int = 0) -> CSRGraph:
    src, dst = uniform_edges(n, m, seed, threads)
    return from_edges(n, src, dst, threads=threads, name=f"uniform-n{n}-m{m}")


def grid3d(X: int, Y: int, Z: int, threads: int = 0) -> CSRGraph:
    src, dst = grid3d_edges(X, Y, Z, threads)
    return from_edges(X * Y * Z, src, dst, threads=threads, name=f"grid3d-{X}x{Y}x{Z}")


def parse_edge_list(text, threads: int = 0, first_line: int = 1):
    """(src, dst, max_id) of a text edge list held in memory (bytes, bytearray, mmap or a
    uint8 array): one "u v" pair per line, ids non-negative decimal integers separated by
    blanks, tabs or a comma; blank lines and lines starting with '#' or '%' are skipped and
    fields after the second id are ignored. Raises ValueError naming the first bad line
    (numbered from ``first_line``)."""
    buf = np.frombuffer(text, dtype=np.uint8) if not isinstance(text, np.ndarray) else text
    n_bytes = int(buf.size)
    addr = buf.ctypes.data if n_bytes else None
    max_id, err = ctypes.c_int64(-1), ctypes.c_int64(-1)
    lib = _load()

    def fail(code: int):
        if code in (-3, -5):
            line = int(np.count_nonzero(buf[: err.value] == 10)) + first_line
            what = "vertex id above 2^31 - 2" if code == -3 else "not a pair of non-negative integer ids"
            raise ValueError(f"edge list line {line}: {what}")
        raise ValueError("gg_parse_edge_list: bad arguments")

    m = lib.gg_parse_edge_list(addr, n_bytes, None, None, 0, ctypes.byref(max_id), ctypes.byref(err), int(threads))
    if m < 0:
        fail(m)
    src = np.empty(max(m, 1), dtype=np.int32)
    dst = np.empty(max(m, 1), dtype=np.int32)
    got = lib.gg_parse_edge_list(addr, n_bytes, _p(src, _P32), _p(dst, _P32), int(m), ctypes.byref(max_id),
                                 ctypes.byref(err), int(threads))
    if got != m:
        fail(got)
    return src[:m], dst[:m], int(max_id.value)


def _line_end(buf, pos: int) -> int:
    """Index of the first newline at or after pos (len(buf) if none)."""
    while pos < buf.size:
        hit = np.flatnonzero(buf[pos: pos + 4096] == 10)
        if hit.size:
            return pos + int(hit[0])
        pos += 4096
    return int(buf.size)


def _parse_matrix_market(buf, threads: int):
    """(src, dst, n) of a MatrixMarket coordinate file: a '%%MatrixMarket matrix coordinate
    ...' header, '%' comment lines, a 'rows cols entries' size line, then one 1-based
    'i j [value...]' entry per line. Rows and columns share one vertex numbering, so
    n = max(rows, cols); values are ignored."""
    end = _line_end(buf, 0)
    head = bytes(buf[:end]).decode("ascii", "replace").split()
    if len(head) < 3 or head[1].lower() != "matrix" or head[2].lower() != "coordinate":
        raise ValueError("MatrixMarket: only 'matrix coordinate' files hold a graph")
    pos, line_no = end + 1, 2
    while pos < buf.size:
        end = _line_end(buf, pos)
        line = bytes(buf[pos:end]).strip()
        if line and not line.startswith(b"%"):
            break
        pos, line_no = end + 1, line_no + 1
    else:
        raise ValueError("MatrixMarket: no size line")
    try:
        rows, cols, entries = (int(x) for x in line.split()[:3])
    except ValueError:
        raise ValueError(f"MatrixMarket line {line_no}: expected 'rows cols entries'") from None
    src, dst, max_id = parse_edge_list(buf[end + 1:], threads, first_line=line_no + 1)
    if src.size != entries:
        raise ValueError(f"MatrixMarket: {src.size} entries, the size line says {entries}")
    if src.size and (min(int(src.min()), int(dst.min())) < 1 or max_id > max(rows, cols)):
        raise ValueError("MatrixMarket: an entry lies outside the 1-based matrix")
    return src - 1, dst - 1, max(rows, cols)


def _parse_graph_text(buf, threads: int):
    """(src, dst, n) of a text edge list or a MatrixMarket coordinate file in buf."""
    if bytes(buf[:14]) == b"%%MatrixMarket":
        return _parse_matrix_market(buf, threads)
    src, dst, max_id = parse_edge_list(buf, threads)
    return src, dst, max_id + 1


def load_edge_list(path: str, compact: bool = False, threads: int = 0, name: str = "") -> CSRGraph:
    """The cleaned symmetric CSR of a graph file: a text edge list (``parse_edge_list``'s
    format, the SNAP form) or a MatrixMarket coordinate file (1-based ids, recognised by its
    header); ``.gz`` files are decompressed. Every pair becomes an undirected edge, as the
    paper treats its inputs (Sec. 4); self-loops and duplicates are removed. Vertex ids are
    the file's (edge list: n = largest id + 1; MatrixMarket: ids - 1, n = the matrix order;
    ids that never appear have degree 0) unless ``compact``, which renumbers the ids that
    appear to 0..n-1 in ascending order and keeps the original (0-based) ids in ``ids``."""
    import gzip
    import mmap

    name = name or os.path.basename(path)
    if path.endswith(".gz"):
        with gzip.open(path, "rb") as f:
            data = np.frombuffer(f.read(), dtype=np.uint8)
        try:
            src, dst, n = _parse_graph_text(data, threads)
        except ValueError as e:
            raise ValueError(f"{path}: {e}") from None
    else:
        with open(path, "rb") as f:
            if os.fstat(f.fileno()).st_size == 0:
                src, dst, n = _parse_graph_text(np.zeros(0, np.uint8), threads)
            else:
                bad = None
                with mmap.mmap(f.fileno(), 0, access=mmap.ACCESS_READ) as mm:
                    buf = np.frombuffer(mm, dtype=np.uint8)
                    try:
                        src, dst, n = _parse_graph_text(buf, threads)
                    except ValueError as e:  # re-raised once the map is closed: the
                        bad = str(e)         # traceback would keep the view alive
                    del buf
                if bad:
                    raise ValueError(f"{path}: {bad}")
    if src.size == 0:
        raise ValueError(f"{path}: no edges")
    if not compact:
        return from_edges(n, src, dst, threads=threads, name=name)
    ids = np.unique(np.concatenate([src, dst]))
    g = from_edges(ids.size, np.searchsorted(ids, src).astype(np.int32), np.searchsorted(ids, dst).astype(np.int32),
                   threads=threads, name=name)
    g.ids = ids
    return g


def pick_roots(g: CSRGraph, k: int, seed: int) -> np.ndarray:
    """k distinct roots with degree > 0, drawn from a seeded counter-based stream."""
    out = np.empty(max(k, 1), dtype=np.int32)
    got = _load().gg_pick_roots(g.n, _p(g.offsets, _P64), int(k), int(seed) & (2**64 - 1), _p(out, _P32))
    if got < 0:
        raise ValueError("gg_pick_roots: bad arguments")
    return out[:got].copy()


def root_seed(graph_seed: int) -> int:
    return graph_seed ^ 0x5EED
