"""Persistent (one-launch) searches and bottom-up levels: same levels as the oracle, valid
parents, same m_c, for every loop mode and direction policy."""
import numpy as np
import pytest

from _graphs import binary_tree_edges, load_golden, path_edges, random_edges, star_edges

pytestmark = pytest.mark.gpu

# (loop mode, bottom-up, alpha, beta)
POLICIES = {
    "persistent-td": (0, 0, 14, 24),
    "persistent-do": (0, 1, 8, 24),
    "persistent-bu-eager": (0, 1, 1 << 20, 1 << 20),  # bottom-up from the first growing level on
    "persistent-bu-flip": (0, 1, 1 << 20, 1),         # bottom-up while growing, top-down once shrinking
}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_1605_gb300 import _build

    _build.build_bfs()
    return torch


def _upload(capi, g, policy, force64=False):
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz,
                              capi.BFS_OFFSETS_INT64 | (capi.BFS_KEEP_INT64 if force64 else 0))
    loop, bu, alpha, beta = POLICIES[policy]
    capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, loop)
    capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, bu)
    capi.bfs_graph_set_option(h, capi.BFS_OPT_ALPHA, alpha)
    capi.bfs_graph_set_option(h, capi.BFS_OPT_BETA, beta)
    return h


def _check(capi, oracle, torch, h, g, root):
    dl = torch.empty(g.n, dtype=torch.int32, device="cuda")
    dp = torch.empty(g.n, dtype=torch.int32, device="cuda")
    st = capi.bfs_run(h, root, dl, dp, want_stats=True)
    lv, pr = dl.cpu().numpy(), dp.cpu().numpy()
    ref, _ = oracle.bfs(g.offsets, g.cols, root)
    assert np.array_equal(lv, ref), f"root {root}: levels differ at {np.flatnonzero(lv != ref)[:8]}"
    code, bad = oracle.check_tree(g.offsets, g.cols, root, ref, lv, pr)
    assert code == 0, (oracle.TREE_CODES[code], bad)
    assert st.edges_traversed == oracle.component_edges(g.offsets, ref)
    assert st.vertices_reached == int((ref >= 0).sum()) and st.depth == int(ref.max()) + 1
    return st


@pytest.mark.parametrize("policy", sorted(POLICIES))
def test_rmat_policies(torch_cuda, oracle_mod, graphs_mod, policy):
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(16, 16, seed=graphs_mod.GRAPH_SEED_BASE)
    roots = graphs_mod.pick_roots(g, 16, graphs_mod.root_seed(graphs_mod.GRAPH_SEED_BASE))
    for force64 in (False, True):
        h = _upload(capi, g, policy, force64)
        try:
            bu_levels = 0
            for r in roots[:8]:
                bu_levels += _check(capi, oracle_mod, torch_cuda, h, g, int(r)).bottom_up_levels
            if POLICIES[policy][1]:
                assert bu_levels > 0
            else:
                assert bu_levels == 0
        finally:
            capi.bfs_graph_destroy(h)


@pytest.mark.parametrize("policy", sorted(POLICIES))
def test_families_policies(torch_cuda, oracle_mod, graphs_mod, policy):
    from paper_1408_1605_gb300 import capi

    fams = [graphs_mod.from_edges(4000, *path_edges(4000)), graphs_mod.from_edges(3000, *star_edges(3000)),
            graphs_mod.from_edges(4095, *binary_tree_edges(4095)), graphs_mod.grid3d(23, 17, 11),
            graphs_mod.uniform(20000, 60000, seed=4)]
    fx = load_golden("two_components.txt")
    fams.append(graphs_mod.from_edges(fx["n"], fx["src"], fx["dst"]))
    rng = np.random.default_rng(6)
    for _ in range(3):
        n = int(rng.integers(2, 300))
        fams.append(graphs_mod.from_edges(n, *random_edges(n, int(rng.integers(0, 4 * n)), rng)))
    for g in fams:
        h = _upload(capi, g, policy)
        try:
            for root in sorted({0, g.n - 1, g.n // 2, int(rng.integers(0, g.n))}):
                _check(capi, oracle_mod, torch_cuda, h, g, root)
        finally:
            capi.bfs_graph_destroy(h)


def test_persistent_host_outputs_and_repeat(torch_cuda, oracle_mod, graphs_mod):
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(15, 16, seed=12)
    h = _upload(capi, g, "persistent-do")
    try:
        for r in graphs_mod.pick_roots(g, 3, 5):
            lv = np.empty(g.n, np.int32)
            pr = np.empty(g.n, np.int32)
            capi.bfs_run(h, int(r), lv, pr)
            ref, _ = oracle_mod.bfs(g.offsets, g.cols, int(r))
            assert np.array_equal(lv, ref)
            assert oracle_mod.check_tree(g.offsets, g.cols, int(r), ref, lv, pr)[0] == 0
    finally:
        capi.bfs_graph_destroy(h)


def test_option_errors(torch_cuda, graphs_mod):
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(8, 8, seed=1)
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64)
    try:
        assert capi.bfs_graph_get_option(h, capi.BFS_OPT_LOOP) == capi.BFS_LOOP_GRAPH
        for opt, val in ((capi.BFS_OPT_LOOP, 7), (capi.BFS_OPT_ALPHA, 0), (capi.BFS_OPT_PERSIST_CTAS, 65), (99, 1)):
            with pytest.raises(capi.BfsError):
                capi.bfs_graph_set_option(h, opt, val)
    finally:
        capi.bfs_graph_destroy(h)


def test_level_profile_matches_oracle_level_sizes(torch_cuda, oracle_mod, graphs_mod):
    """The per-level profile of a persistent search lists, for level i, the size of the
    frontier it expanded: the number of vertices at hop distance i."""
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(16, 16, seed=17)
    r = int(graphs_mod.pick_roots(g, 1, 2)[0])
    for policy in ("persistent-td", "persistent-do"):
        h = _upload(capi, g, policy)
        try:
            st = _check(capi, oracle_mod, torch_cuda, h, g, r)
            prof = capi.bfs_level_profile(h)
            ref, _ = oracle_mod.bfs(g.offsets, g.cols, r)
            assert len(prof) == st.depth
            assert [p["frontier"] for p in prof] == np.bincount(ref[ref >= 0]).tolist()
            assert sum(p["bottom_up"] for p in prof) == st.bottom_up_levels
            assert all(p["ms"] >= 0 for p in prof) and sum(p["ms"] for p in prof) <= st.device_ms + 0.05
        finally:
            capi.bfs_graph_destroy(h)


def test_barrier_wait_expiry_reports_timeout(torch_cuda, oracle_mod, graphs_mod):
    """Failure detection without a fault: with a wait limit of 0 every grid-barrier wait but
    the last arrival's gives up at once, the search stops and bfs_run reports
    BFS_ERR_TIMEOUT; the same graph then searches correctly with the default limit."""
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(14, 16, seed=23)
    r = int(graphs_mod.pick_roots(g, 1, 4)[0])
    h = _upload(capi, g, "persistent-td")
    try:
        default = capi.bfs_graph_get_option(h, capi.BFS_OPT_WAIT_LIMIT)
        capi.bfs_graph_set_option(h, capi.BFS_OPT_WAIT_LIMIT, 0)
        lv = torch_cuda.empty(g.n, dtype=torch_cuda.int32, device="cuda")
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_run(h, r, lv, lv.clone(), want_stats=True)
        assert e.value.status == 5  # BFS_ERR_TIMEOUT
        capi.bfs_graph_set_option(h, capi.BFS_OPT_WAIT_LIMIT, default)
        _check(capi, oracle_mod, torch_cuda, h, g, r)
    finally:
        capi.bfs_graph_destroy(h)


@pytest.mark.parametrize("ctas", [1, 2])
def test_few_ctas_per_sm(torch_cuda, oracle_mod, graphs_mod, ctas):
    """A persistent search with BFS_OPT_PERSIST_CTAS set (fewer, larger level boundaries)
    returns the same BFS, top-down and direction-optimizing."""
    from paper_1408_1605_gb300 import capi

    for g in (graphs_mod.rmat(15, 16, seed=29), graphs_mod.grid3d(21, 19, 17)):
        for policy in ("persistent-td", "persistent-do"):
            h = _upload(capi, g, policy)
            try:
                capi.bfs_graph_set_option(h, capi.BFS_OPT_PERSIST_CTAS, ctas)
                assert capi.bfs_graph_get_option(h, capi.BFS_OPT_PERSIST_CTAS) == ctas
                for root in (0, g.n // 3, g.n - 1):
                    _check(capi, oracle_mod, torch_cuda, h, g, root)
            finally:
                capi.bfs_graph_destroy(h)
