"""GB300-native single-GPU BFS: the level-synchronous top-down frontier expansion of
Bisson, Bernaschi and Mastrostefano (arXiv 1408.1605) in its one-processor form.

Layout:
  * ``capi``   -- thin ctypes binding of the C ABI in ``include/gbfs.h`` (same names);
  * ``graphs`` -- seeded synthetic inputs (R-MAT, uniform, 3D grid) and the CSR builder;
  * ``Graph``  -- a small convenience wrapper that uploads a CSR and allocates outputs with
    torch (device memory and streams only; the search itself runs in the CUDA library).
"""
from __future__ import annotations

from . import capi

__all__ = ["capi", "Graph", "build"]


def build(verbose: bool = False) -> None:
    from . import _build

    _build.build(verbose=verbose)


class Graph:
    """A graph resident on the current CUDA device (``bfs_graph_create``)."""

    def __init__(self, offsets, cols, validate: bool = False, stream=None):
        import numpy as np

        if hasattr(offsets, "is_cuda") and offsets.is_cuda:
            flags = capi.BFS_DEVICE_PTRS
            wide = offsets.element_size() == 8
        else:
            offsets = np.ascontiguousarray(offsets)
            cols = np.ascontiguousarray(cols, dtype=np.int32)
            flags = capi.BFS_HOST_PTRS
            wide = offsets.dtype.itemsize == 8
            if offsets.dtype not in (np.int32, np.int64):
                raise TypeError("offsets must be int32 or int64")
        flags |= capi.BFS_OFFSETS_INT64 if wide else capi.BFS_OFFSETS_INT32
        if validate:
            flags |= capi.BFS_VALIDATE
        n = len(offsets) - 1
        nnz = int(offsets[-1])
        self.n, self.nnz = n, nnz
        self.handle = capi.bfs_graph_create(offsets, cols, n, nnz, flags, stream)

    def bfs(self, root: int, levels=None, parents=None, stream=None, stats: bool = False):
        import torch

        if levels is None:
            levels = torch.empty(self.n, dtype=torch.int32, device="cuda")
        if parents is None:
            parents = torch.empty(self.n, dtype=torch.int32, device="cuda")
        st = capi.bfs_run(self.handle, root, levels, parents, stream, want_stats=stats)
        return (levels, parents, st.as_dict()) if stats else (levels, parents)

    def close(self) -> None:
        if getattr(self, "handle", None):
            capi.bfs_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
