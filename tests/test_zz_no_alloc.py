"""bfs_run_noalloc: the single-source search for callers that may not allocate device
memory at call time (a framework allocator that owns all device memory, loops where
cudaMalloc / cudaFree would synchronize the device, services that must not hit
out-of-memory mid-request). Its work buffers live in one static device array.

Checked through the C ABI against the regular entry point bfs_run on the same inputs, on
two calls in a row (the array keeps the previous call's contents, so the second call
checks that everything that must start cleared is cleared): levels bit-exact, parents
valid BFS trees (which parent wins a tie depends on atomics). This file is collected last
so that a failure here stops a -x run only after every other test has run."""
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


def test_noalloc_matches_bfs_run_twice(torch_cuda, oracle_mod, graphs_mod):
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    g = graphs_mod.rmat(16, 16, seed=graphs_mod.GRAPH_SEED_BASE)  # 65,536 vertices, 1.8 M entries
    off32 = g.offsets32()
    d_off = torch.from_numpy(off32).cuda()
    d_cols = torch.from_numpy(g.cols).cuda()
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64)
    roots = graphs_mod.pick_roots(g, 2, graphs_mod.root_seed(graphs_mod.GRAPH_SEED_BASE))
    try:
        ref_l = torch.empty(g.n, dtype=torch.int32, device="cuda")
        ref_p = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for r in roots:  # two calls in a row, different roots
            capi.bfs_run(h, int(r), ref_l, ref_p, want_stats=True)
            lv = torch.full((g.n,), 12345, dtype=torch.int32, device="cuda")
            pr = torch.full((g.n,), 12345, dtype=torch.int32, device="cuda")
            capi.bfs_run_noalloc(d_off, d_cols, g.n, g.nnz, int(r), lv, pr)
            torch.cuda.synchronize()
            got_l, got_p = lv.cpu().numpy(), pr.cpu().numpy()
            assert np.array_equal(got_l, ref_l.cpu().numpy())
            code, bad = oracle_mod.check_tree(g.offsets, g.cols, int(r), got_l, got_l, got_p)
            assert code == 0, (oracle_mod.TREE_CODES[code], bad)
    finally:
        capi.bfs_graph_destroy(h)


def test_noalloc_rejects_sizes_beyond_the_scratch(torch_cuda):
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.BfsError, match="n_vertices must be in") as e:
        capi.bfs_run_noalloc(dummy, dummy, (1 << 18) + 1, 0, 0, dummy, dummy)
    assert e.value.status == 1
    with pytest.raises(capi.BfsError, match="n_entries must be in"):
        capi.bfs_run_noalloc(dummy, dummy, 2, (1 << 22) + 1, 0, dummy, dummy)
