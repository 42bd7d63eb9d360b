"""Parity of the multi-source (batched) search with the oracle: every root's slice of a
64-root wave has exactly the single-source levels, valid parents, and the oracle's m_c."""

import numpy as np
import pytest

from _graphs import binary_tree_edges, load_golden, path_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_1605_gb300 import _build

    _build.build_bfs()
    return torch


def _upload(capi, g, force64=False, host_loop=False):
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz,
                              capi.BFS_OFFSETS_INT64 | (capi.BFS_KEEP_INT64 if force64 else 0))
    if host_loop:
        capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, capi.BFS_LOOP_HOST)
    return h


def check_wave(capi, oracle, torch, h, g, roots, host_out=False):
    roots = np.asarray(roots, dtype=np.int32)
    k = roots.size
    if host_out:
        lv = np.empty((k, g.n), dtype=np.int32)
        pr = np.empty((k, g.n), dtype=np.int32)
        st = capi.bfs_run_batch(h, roots, lv, pr, want_stats=True)
    else:
        dl = torch.empty((k, g.n), dtype=torch.int32, device="cuda")
        dp = torch.empty((k, g.n), dtype=torch.int32, device="cuda")
        st = capi.bfs_run_batch(h, roots, dl, dp, want_stats=True)
        lv, pr = dl.cpu().numpy(), dp.cpu().numpy()
    for b, r in enumerate(roots.tolist()):
        ref, _ = oracle.bfs(g.offsets, g.cols, r)
        assert np.array_equal(lv[b], ref), f"root slot {b} ({r}): levels differ at {np.flatnonzero(lv[b] != ref)[:8]}"
        code, bad = oracle.check_tree(g.offsets, g.cols, r, ref, lv[b], pr[b])
        assert code == 0, (b, r, oracle.TREE_CODES[code], bad)
        assert st[b].edges_traversed == oracle.component_edges(g.offsets, ref)
        assert st[b].vertices_reached == int((ref >= 0).sum())
        assert st[b].depth == int(ref.max()) + 1
    return st


@pytest.mark.parametrize("force64", [False, True])
def test_rmat16_wave_of_64(torch_cuda, oracle_mod, graphs_mod, force64):
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(16, 16, seed=graphs_mod.GRAPH_SEED_BASE)
    roots = graphs_mod.pick_roots(g, 64, 11)
    h = _upload(capi, g, force64)
    try:
        check_wave(capi, oracle_mod, torch_cuda, h, g, roots)
        check_wave(capi, oracle_mod, torch_cuda, h, g, roots[:17])  # ragged wave, reused buffers
    finally:
        capi.bfs_graph_destroy(h)


def test_wave_sizes_duplicates_components(torch_cuda, oracle_mod, graphs_mod):
    from paper_1408_1605_gb300 import capi

    fx = load_golden("two_components.txt")
    g = graphs_mod.from_edges(fx["n"], fx["src"], fx["dst"])
    h = _upload(capi, g)
    try:
        check_wave(capi, oracle_mod, torch_cuda, h, g, [0])
        check_wave(capi, oracle_mod, torch_cuda, h, g, list(range(12)))  # every vertex, isolated 11 too
        check_wave(capi, oracle_mod, torch_cuda, h, g, [3, 3, 8, 11, 3, 0])  # repeats
        check_wave(capi, oracle_mod, torch_cuda, h, g, [5] * 64)
    finally:
        capi.bfs_graph_destroy(h)


def test_grid_tree_path_waves(torch_cuda, oracle_mod, graphs_mod):
    from paper_1408_1605_gb300 import capi

    rng = np.random.default_rng(3)
    for g in (graphs_mod.grid3d(21, 17, 13), graphs_mod.from_edges(2047, *binary_tree_edges(2047)),
              graphs_mod.from_edges(3000, *path_edges(3000))):
        h = _upload(capi, g)
        try:
            check_wave(capi, oracle_mod, torch_cuda, h, g, rng.integers(0, g.n, 64))
        finally:
            capi.bfs_graph_destroy(h)


def test_host_loop_and_host_outputs(torch_cuda, oracle_mod, graphs_mod):
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(14, 16, seed=31)
    roots = graphs_mod.pick_roots(g, 40, 2)
    for host_loop in (False, True):
        h = _upload(capi, g, host_loop=host_loop)
        try:
            check_wave(capi, oracle_mod, torch_cuda, h, g, roots, host_out=True)
            check_wave(capi, oracle_mod, torch_cuda, h, g, roots[:9], host_out=False)
        finally:
            capi.bfs_graph_destroy(h)


def test_batch_matches_single_source(torch_cuda, oracle_mod, graphs_mod):
    """A root alone (bfs_run) and inside a wave give identical levels."""
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    g = graphs_mod.rmat(18, 16, seed=77)
    roots = graphs_mod.pick_roots(g, 64, 5)
    h = _upload(capi, g)
    try:
        dl = torch.empty((64, g.n), dtype=torch.int32, device="cuda")
        dp = torch.empty((64, g.n), dtype=torch.int32, device="cuda")
        capi.bfs_run_batch(h, roots, dl, dp)
        sl = torch.empty(g.n, dtype=torch.int32, device="cuda")
        sp = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for b in (0, 31, 63):
            capi.bfs_run(h, int(roots[b]), sl, sp)
            assert torch.equal(sl, dl[b])
    finally:
        capi.bfs_graph_destroy(h)


def test_batch_errors(torch_cuda, graphs_mod):
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(10, 8, seed=1)
    h = _upload(capi, g)
    out = torch_cuda.empty((65, g.n), dtype=torch_cuda.int32, device="cuda")
    try:
        for roots in ([], list(range(65)), [0, g.n], [-1]):
            with pytest.raises(capi.BfsError) as e:
                capi.bfs_run_batch(h, np.array(roots, dtype=np.int32), out, out)
            assert e.value.status == 1
    finally:
        capi.bfs_graph_destroy(h)


# (bottom-up, alpha, beta): Beamer's defaults, bottom-up from the first growing level, and
# bottom-up while growing / top-down once shrinking
BU_POLICIES = {"do": (1, 8, 24), "bu-eager": (1, 1 << 20, 1 << 20), "bu-flip": (1, 1 << 20, 1)}


@pytest.mark.parametrize("policy", sorted(BU_POLICIES))
@pytest.mark.parametrize("relabel", [False, True])
def test_waves_with_bottom_up_levels(torch_cuda, oracle_mod, graphs_mod, policy, relabel):
    """Waves that run some levels bottom-up (each vertex pulls the bits it misses from its
    neighbours' frontier masks) give every root the single-source levels and valid parents."""
    from paper_1408_1605_gb300 import capi

    bu, alpha, beta = BU_POLICIES[policy]
    gs = [graphs_mod.rmat(15, 16, seed=19), graphs_mod.grid3d(15, 13, 11), graphs_mod.uniform(12000, 48000, seed=3),
          graphs_mod.from_edges(3000, *path_edges(3000))]
    fx = load_golden("two_components.txt")
    gs.append(graphs_mod.from_edges(fx["n"], fx["src"], fx["dst"]))
    flags = capi.BFS_OFFSETS_INT64 | (capi.BFS_RELABEL_DEGREE if relabel else 0)
    for g in gs:
        rng = np.random.default_rng(g.n + 11)
        h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, flags)
        try:
            capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, bu)
            capi.bfs_graph_set_option(h, capi.BFS_OPT_ALPHA, alpha)
            capi.bfs_graph_set_option(h, capi.BFS_OPT_BETA, beta)
            roots = rng.integers(0, g.n, size=min(64, g.n))
            roots[1] = roots[0]  # a repeated root
            st = check_wave(capi, oracle_mod, torch_cuda, h, g, roots)
            if g.name.startswith("rmat") and policy != "do":
                assert st[0].bottom_up_levels > 0
            check_wave(capi, oracle_mod, torch_cuda, h, g, roots[:5], host_out=True)
        finally:
            capi.bfs_graph_destroy(h)


@pytest.mark.parametrize("dense_rows", [-1, 1, 0, 1 << 20])
@pytest.mark.parametrize("bottom_up", [0, 1])
def test_claims_beyond_the_event_slots(torch_cuda, oracle_mod, graphs_mod, bottom_up, dense_rows):
    """Hub vertices claimed by many frontier vertices with disjoint root bits: roots at the
    leaves of a star (every leaf's edge claims its own bits of the centre, up to 64 claims at
    one vertex in one level), and a second hub joined to every leaf. Claims of one root bit
    are written at once; with each leaf holding two roots (repeated roots), every claim
    carries two bits and the wave's records spill past the per-vertex slots: into dense rows
    (the default pool, one row, none, a row per vertex), then the overflow list. Every root
    still gets the oracle's levels and a valid tree."""
    from paper_1408_1605_gb300 import capi

    leaves = np.arange(1, 65, dtype=np.int32)
    src = np.concatenate([np.zeros(64, np.int32), np.full(64, 65, np.int32), np.arange(65, 164, dtype=np.int32)])
    dst = np.concatenate([leaves, leaves, np.arange(66, 165, dtype=np.int32)])  # hub 65 leads into a path
    g = graphs_mod.from_edges(165, src, dst)
    for flags in (0, capi.BFS_RELABEL_DEGREE):
        h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64 | flags)
        try:
            capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, bottom_up)
            capi.bfs_graph_set_option(h, capi.BFS_OPT_WAVE_DENSE_ROWS, dense_rows)
            check_wave(capi, oracle_mod, torch_cuda, h, g, leaves)
            check_wave(capi, oracle_mod, torch_cuda, h, g, np.repeat(leaves[:32], 2))
            check_wave(capi, oracle_mod, torch_cuda, h, g, np.concatenate([leaves[:32], [0, 65] * 16]))
            check_wave(capi, oracle_mod, torch_cuda, h, g, leaves[::-1].copy(), host_out=True)
        finally:
            capi.bfs_graph_destroy(h)


@pytest.mark.parametrize("shape", list(range(9)))
@pytest.mark.parametrize("force64", [False, True])
def test_every_batch_shape(torch_cuda, oracle_mod, graphs_mod, shape, force64):
    """Every compiled batched shape (CTA tiles and warp tiles), both offset widths, on R-MAT
    (input order and degree-relabelled), a grid, a uniform multigraph-free graph and a graph
    with an isolated vertex, top-down waves and waves with bottom-up levels; every slot has
    the oracle's levels and a valid tree."""
    from paper_1408_1605_gb300 import capi

    fx = load_golden("two_components.txt")
    gs = [(graphs_mod.rmat(15, 16, seed=23), 0), (graphs_mod.rmat(15, 16, seed=23), capi.BFS_RELABEL_DEGREE),
          (graphs_mod.grid3d(13, 11, 9), 0), (graphs_mod.uniform(12000, 60000, seed=4), 0),
          (graphs_mod.from_edges(fx["n"], fx["src"], fx["dst"]), 0)]
    for g, relabel in gs:
        rng = np.random.default_rng(g.n + shape)
        roots = rng.integers(0, g.n, size=min(64, g.n))
        roots[2] = roots[1]  # a repeated root
        h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64 | relabel
                                  | (capi.BFS_KEEP_INT64 if force64 else 0))
        try:
            capi.bfs_graph_set_shape(h, capi.BFS_KERNEL_BATCH, shape)
            check_wave(capi, oracle_mod, torch_cuda, h, g, roots)
            check_wave(capi, oracle_mod, torch_cuda, h, g, roots[:7])
            capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, 1)
            check_wave(capi, oracle_mod, torch_cuda, h, g, roots)
        finally:
            capi.bfs_graph_destroy(h)
