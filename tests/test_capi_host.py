"""The C-ABI library builds for sm_103a, loads, exports every function include/gbfs.h
declares, and rejects bad arguments on the host before touching a GPU (CPU only)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def capi():
    from paper_1408_1605_gb300 import _build, capi

    _build.build_bfs()
    return capi


def test_exports_every_declared_symbol(capi):
    names = capi.declared_functions()
    assert "bfs_graph_create" in names and "bfs_run" in names and "bfs_expand" in names
    L = ctypes.CDLL(capi.library_path())
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    unbound = [n for n in names if not callable(getattr(capi, n, None))]
    assert not unbound, unbound  # the binding has a function of the same name for each


def test_version(capi):
    assert "sm_103a" in capi.bfs_version()


def _create(capi, off, cols, n, nnz, flags):
    out = ctypes.c_void_p()
    s = capi.lib().bfs_graph_create(capi.ptr(off), capi.ptr(cols), n, nnz, flags, 0, ctypes.byref(out))
    return s, out.value


def test_create_rejects_bad_arguments(capi):
    off = np.array([0, 1, 2], dtype=np.int32)
    cols = np.array([1, 0], dtype=np.int32)
    L = capi.lib()
    assert L.bfs_graph_create(capi.ptr(off), capi.ptr(cols), 2, 2, 0, 0, None) == 1  # out NULL
    assert _create(capi, None, cols, 2, 2, 0)[0] == 1
    assert _create(capi, off, None, 2, 2, 0)[0] == 1
    assert _create(capi, off, cols, 0, 2, 0)[0] == 1
    assert _create(capi, off, cols, 2, -1, 0)[0] == 1
    assert _create(capi, off, cols, 2, 2, 0x1000)[0] == 1
    assert _create(capi, off, cols, 2, 2, capi.BFS_HOST_PTRS | capi.BFS_DEVICE_PTRS)[0] == 1
    assert _create(capi, off, cols, 2, 2, capi.BFS_OFFSETS_INT32 | capi.BFS_OFFSETS_INT64)[0] == 1
    assert "both set" in capi.bfs_last_error()


def test_create_rejects_malformed_csr(capi):
    cols = np.array([1, 0], dtype=np.int32)
    for off in ([1, 1, 2], [0, 2, 1], [0, 1, 3]):
        s, _ = _create(capi, np.array(off, dtype=np.int32), cols, 2, 2, 0)
        assert s == 2, off
    s, _ = _create(capi, np.array([0, 1, 2], dtype=np.int64), cols, 2, 2, capi.BFS_OFFSETS_INT64)
    assert s != 2  # well-formed: fails later only for want of a GPU, or succeeds on one
    bad_cols = np.array([1, 5], dtype=np.int32)
    s, _ = _create(capi, np.array([0, 1, 2], dtype=np.int32), bad_cols, 2, 2, capi.BFS_VALIDATE)
    assert s == 2 and "out of range" in capi.bfs_last_error()
    asym = np.array([1, 1], dtype=np.int32)  # 0->1, 1->1 : not symmetric
    s, _ = _create(capi, np.array([0, 1, 2], dtype=np.int32), asym, 2, 2, capi.BFS_VALIDATE)
    assert s == 2 and "symmetric" in capi.bfs_last_error()


def test_calls_reject_null_graph(capi):
    L = capi.lib()
    lv = np.zeros(4, dtype=np.int32)
    assert L.bfs_run(None, 0, capi.ptr(lv), capi.ptr(lv), None, None) == 1
    assert L.bfs_expand(None, None, 0, 1, None, None, None, None, None, None) == 1
    assert L.bfs_graph_info(None, None, None) == 1
    assert L.bfs_graph_destroy(None) == 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1408_1605_gb300 import _build, capi

    monkeypatch.setattr(_build, "LIB_BFS", str(tmp_path / "missing.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        capi.lib()


def test_serve_host_side_checks(capi):
    """Server creation, lookups and reports need no GPU."""
    with pytest.raises(capi.BfsError) as e:
        capi.bfs_serve_create(max_wave=65)
    assert e.value.status == 1
    srv = capi.bfs_serve_create(memory_cap_bytes=1 << 20, max_wave=8, queue_capacity=4)
    try:
        buf = np.zeros(4, dtype=np.int32)
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_serve_submit(srv, 0, 0, buf, buf)
        assert e.value.status == 8
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_serve_wait(srv, 1, 0)
        assert e.value.status == 8
        rep = capi.bfs_serve_stats(srv)
        assert rep["submitted"] == 0 and rep["completed"] == 0
    finally:
        capi.bfs_serve_destroy(srv)
    assert capi.lib().bfs_serve_destroy(None) == 0


def test_shape_tables(capi):
    for kind in (capi.BFS_KERNEL_SINGLE, capi.BFS_KERNEL_BATCH):
        n = capi.bfs_shape_count(kind)
        assert n >= 2
        for s in range(n):
            info = capi.bfs_shape_info(kind, s)
            assert info["block"] % 32 == 0 and info["edges_per_thread"] >= 1
            tile = (32 if info["warp_tiles"] else info["block"]) * info["edges_per_thread"]
            assert info["claim_buffer"] >= tile and tile % 128 == 0
            assert info["warp_tiles"] in (0, 1)
    assert capi.bfs_shape_count(7) == 0
    # tests/test_gpu_bfs.py runs every single-source shape: keep its list in step
    assert capi.bfs_shape_count(capi.BFS_KERNEL_SINGLE) == 10
    with pytest.raises(capi.BfsError):
        capi.bfs_shape_info(0, 99)


def test_autotune_cache_roundtrip(capi, monkeypatch, tmp_path):
    """Tunes once per key, then applies the cached shape without timing again."""
    from paper_1408_1605_gb300 import autotune

    monkeypatch.setenv("GBFS_TUNE_CACHE", str(tmp_path / "tune.json"))
    calls = {"tune": 0, "set": []}

    def fake_tune(graph, kind, roots, levels, parents, stream=None):
        calls["tune"] += 1
        return 1, [3.0, 1.0]

    monkeypatch.setattr(capi, "bfs_tune", fake_tune)
    monkeypatch.setattr(capi, "bfs_graph_set_shape", lambda g, k, s: calls["set"].append((k, s)))
    monkeypatch.setattr(capi, "bfs_graph_set_option", lambda g, o, v: calls["set"].append(("opt", o, v)))
    monkeypatch.setattr(capi, "bfs_graph_get_option", lambda g, o: 0)
    r1 = autotune.apply_or_tune(0, capi.BFS_KERNEL_SINGLE, "rmat", 1 << 20, [1], None, None)
    assert r1["shape"] == 1 and not r1["cached"] and calls["tune"] == 1
    r2 = autotune.apply_or_tune(0, capi.BFS_KERNEL_SINGLE, "rmat", (1 << 20) + 5, [1], None, None)
    assert r2["cached"] and calls["tune"] == 1 and (0, 1) in calls["set"]
    r3 = autotune.apply_or_tune(0, capi.BFS_KERNEL_BATCH, "rmat", 1 << 20, [1], None, None)
    assert not r3["cached"] and calls["tune"] == 2
    assert autotune.key(0, "grid", 1 << 24, "X") == "X|single|grid|s24"


def test_binding_checks_output_buffers(capi, monkeypatch):
    """Outputs must be contiguous int32 arrays large enough for the call: a wrong buffer
    raises on the host, before any library call could write past it."""
    with pytest.raises(ValueError, match="contiguous"):
        capi.ptr(np.zeros((4, 4), np.int32)[:, 1])
    with pytest.raises(ValueError, match="int32"):
        capi.bfs_run(0, 0, np.zeros(10, np.int64), np.zeros(10, np.int32))
    monkeypatch.setattr(capi, "bfs_graph_info", lambda graph: (10, 20))
    with pytest.raises(ValueError, match="holds 9 entries"):
        capi.bfs_run(0, 0, np.zeros(10, np.int32), np.zeros(9, np.int32))
    with pytest.raises(ValueError, match="holds 19 entries"):
        capi.bfs_run_batch(0, [1, 2], np.zeros((2, 10), np.int32), np.zeros(19, np.int32))
    with pytest.raises(ValueError, match="int32"):
        capi.bfs_serve_submit(0, 0, 0, np.zeros(10, np.float32), np.zeros(10, np.int32))
    with pytest.raises(ValueError, match="holds 9 entries"):
        capi.bfs_tune(0, capi.BFS_KERNEL_SINGLE, [1], np.zeros(9, np.int32), np.zeros(10, np.int32))
    with pytest.raises(ValueError, match="holds 20 entries, the call writes 30"):
        capi.bfs_tune(0, capi.BFS_KERNEL_BATCH, [1, 2, 3], np.zeros((2, 10), np.int32), np.zeros(30, np.int32))


def test_noalloc_checks_its_arrays(capi):
    """bfs_run_noalloc reads and writes its four arrays directly on the device: the binding
    refuses wrong types and sizes, and the library refuses host memory with
    BFS_ERR_INVALID_ARG before any GPU work."""
    off = np.array([0, 1, 2], dtype=np.int32)
    cols = np.array([1, 0], dtype=np.int32)
    lv = np.zeros(2, dtype=np.int32)
    with pytest.raises(ValueError, match="row_offsets holds 2 entries"):
        capi.bfs_run_noalloc(off[:2].copy(), cols, 2, 2, 0, lv, lv)
    with pytest.raises(ValueError, match="row_offsets must be int32"):
        capi.bfs_run_noalloc(off.astype(np.int64), cols, 2, 2, 0, lv, lv)
    with pytest.raises(ValueError, match="cols holds 1 entries"):
        capi.bfs_run_noalloc(off, cols[:1].copy(), 2, 2, 0, lv, lv)
    with pytest.raises(ValueError, match="levels holds 1 entries"):
        capi.bfs_run_noalloc(off, cols, 2, 2, 0, lv[:1].copy(), lv)
    with pytest.raises(ValueError, match="parents must be int32"):
        capi.bfs_run_noalloc(off, cols, 2, 2, 0, lv, np.zeros(2, np.int64))
    L = capi.lib()
    s = L.bfs_run_noalloc(capi.ptr(off), capi.ptr(cols), 2, 2, 0, capi.ptr(lv), capi.ptr(lv), None)
    assert s == 1 and "must be device memory" in capi.bfs_last_error()
