"""bfs_run_noalloc: the single-source search for callers that may not allocate device
memory at call time (a framework allocator that owns all device memory, loops where
cudaMalloc / cudaFree would synchronize the device, services that must not hit
out-of-memory mid-request). Its work buffers live in one static device array.

Checked through the C ABI on two calls in a row (the array keeps the previous call's
contents, so the second call checks that everything that must start cleared is cleared):
levels equal to the oracle's and to the regular entry point bfs_run's on the same inputs,
parents a valid BFS tree for the oracle's levels (which parent wins a tie depends on
atomics). Malformed offsets and an out-of-range column id are refused with
BFS_ERR_INVALID_GRAPH, and the array is still usable afterwards. This file is collected
last so that a failure here stops a -x run only after every other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_1605_gb300 import _build

    _build.build_bfs()
    return torch


def test_noalloc_matches_oracle_and_bfs_run_twice(torch_cuda, oracle_mod, graphs_mod):
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    g = graphs_mod.rmat(16, 16, seed=graphs_mod.GRAPH_SEED_BASE)  # 65,536 vertices, 1.8 M entries
    d_off = torch.from_numpy(g.offsets32()).cuda()
    d_cols = torch.from_numpy(g.cols).cuda()
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64)
    roots = graphs_mod.pick_roots(g, 2, graphs_mod.root_seed(graphs_mod.GRAPH_SEED_BASE))
    try:
        ref_l = torch.empty(g.n, dtype=torch.int32, device="cuda")
        ref_p = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for r in roots:  # two calls in a row, different roots
            want, _ = oracle_mod.bfs(g.offsets, g.cols, int(r))
            capi.bfs_run(h, int(r), ref_l, ref_p, want_stats=True)
            lv = torch.full((g.n,), 12345, dtype=torch.int32, device="cuda")
            pr = torch.full((g.n,), 12345, dtype=torch.int32, device="cuda")
            capi.bfs_run_noalloc(d_off, d_cols, g.n, g.nnz, int(r), lv, pr)
            torch.cuda.synchronize()
            got_l, got_p = lv.cpu().numpy(), pr.cpu().numpy()
            assert np.array_equal(got_l, want)
            assert np.array_equal(got_l, ref_l.cpu().numpy())
            code, bad = oracle_mod.check_tree(g.offsets, g.cols, int(r), want, got_l, got_p)
            assert code == 0, (oracle_mod.TREE_CODES[code], bad)
    finally:
        capi.bfs_graph_destroy(h)


def test_noalloc_refuses_malformed_graphs(torch_cuda, oracle_mod):
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    path_off = np.array([0, 1, 3, 5, 6], dtype=np.int32)  # path 0-1-2-3
    path_cols = np.array([1, 0, 2, 1, 3, 2], dtype=np.int32)
    lv = torch.empty(4, dtype=torch.int32, device="cuda")
    pr = torch.empty(4, dtype=torch.int32, device="cuda")
    bad_off = torch.tensor([0, 3, 1, 5, 6], dtype=torch.int32, device="cuda")  # not monotone
    with pytest.raises(capi.BfsError) as e:
        capi.bfs_run_noalloc(bad_off, torch.from_numpy(path_cols).cuda(), 4, 6, 0, lv, pr)
    assert e.value.status == 2
    bad_cols = torch.tensor([1, 0, 2, 1, 4, 2], dtype=torch.int32, device="cuda")  # id 4 == n
    with pytest.raises(capi.BfsError) as e:
        capi.bfs_run_noalloc(torch.from_numpy(path_off).cuda(), bad_cols, 4, 6, 0, lv, pr)
    assert e.value.status == 2
    # the shared array is usable again after both refusals
    capi.bfs_run_noalloc(torch.from_numpy(path_off).cuda(), torch.from_numpy(path_cols).cuda(), 4, 6, 0, lv, pr)
    torch.cuda.synchronize()
    want, _ = oracle_mod.bfs(path_off.astype(np.int64), path_cols, 0)
    assert np.array_equal(lv.cpu().numpy(), want)


def test_noalloc_rejects_sizes_beyond_the_scratch(torch_cuda):
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    L = capi.lib()
    p = capi.ptr(dummy)
    assert L.bfs_run_noalloc(p, p, (1 << 18) + 1, 0, 0, p, p, None) == 1
    assert "n_vertices must be in" in capi.bfs_last_error()
    assert L.bfs_run_noalloc(p, p, 2, (1 << 22) + 1, 0, p, p, None) == 1
    assert "n_entries must be in" in capi.bfs_last_error()
