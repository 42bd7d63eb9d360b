"""Seeded input generators and the CSR builder (CPU only)."""
import numpy as np
import pytest

from _graphs import random_edges


def _csr_reference(n, src, dst):
    """numpy statement of the builder's contract: symmetric, loop-free, deduplicated,
    rows sorted ascending."""
    keep = src != dst
    a = np.concatenate([src[keep], dst[keep]]).astype(np.int64)
    b = np.concatenate([dst[keep], src[keep]]).astype(np.int64)
    key = np.unique(a * n + b)
    rows, cols = key // n, key % n
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.add.at(offsets, rows + 1, 1)
    return np.cumsum(offsets), cols.astype(np.int32)


@pytest.mark.parametrize("seed", range(6))
def test_builder_matches_reference(graphs_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    src, dst = random_edges(n, int(rng.integers(0, 2000)), rng)
    g = graphs_mod.from_edges(n, src, dst)
    off, cols = _csr_reference(n, src, dst)
    assert np.array_equal(g.offsets, off) and np.array_equal(g.cols, cols)


@pytest.mark.parametrize("n,threads", [(4097, 1), (4097, 7), (50001, 3), (1 << 16, 8)])
def test_builder_many_buckets(graphs_mod, n, threads):
    """Above 4096 vertices the builder groups rows into buckets of several vertices, the
    last one ragged; with hub endpoints, loops and repeats the result still equals the
    contract for any thread count."""
    rng = np.random.default_rng(n + threads)
    src, dst = random_edges(n, 6 * n, rng)
    hubs = rng.integers(0, n, 5).astype(np.int32)
    src[: 2 * n] = hubs[rng.integers(0, 5, 2 * n)]  # skewed sources
    src[-50:], dst[-50:] = n - 1, n - 1              # loops at the last vertex
    g = graphs_mod.from_edges(n, src, dst, threads=threads)
    off, cols = _csr_reference(n, src, dst)
    assert np.array_equal(g.offsets, off) and np.array_equal(g.cols, cols)


def test_builder_rejects_out_of_range(graphs_mod):
    with pytest.raises(ValueError):
        graphs_mod.from_edges(4, np.array([0, 5], np.int32), np.array([1, 1], np.int32))


def test_builder_empty(graphs_mod):
    g = graphs_mod.from_edges(3, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.nnz == 0 and list(g.offsets) == [0, 0, 0, 0]


def _is_clean_symmetric(g):
    off, cols = g.offsets, g.cols
    assert off[0] == 0 and np.all(np.diff(off) >= 0) and off[-1] == cols.size
    rows = np.repeat(np.arange(g.n), np.diff(off))
    assert np.all(rows != cols)
    same_row = rows[1:] == rows[:-1]
    assert np.all(cols[1:][same_row] > cols[:-1][same_row])  # sorted, no duplicates
    fwd = np.sort(rows.astype(np.int64) * g.n + cols)
    bwd = np.sort(cols.astype(np.int64) * g.n + rows)
    assert np.array_equal(fwd, bwd)


def test_rmat_shape_and_cleaning(graphs_mod):
    src, dst = graphs_mod.rmat_edges(12, 16, seed=3)
    assert src.size == 16 * 4096 and src.min() >= 0 and src.max() < 4096 and dst.max() < 4096
    g = graphs_mod.from_edges(4096, src, dst)
    _is_clean_symmetric(g)
    d = g.degrees()
    assert d.max() > 20 * max(1.0, np.median(d[d > 0]))  # heavy-tailed degrees


def test_rmat_deterministic_across_threads(graphs_mod):
    a = graphs_mod.rmat(13, 16, seed=11, threads=1)
    b = graphs_mod.rmat(13, 16, seed=11, threads=5)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.cols, b.cols)
    c = graphs_mod.rmat(13, 16, seed=12)
    assert not np.array_equal(a.cols[:1000], c.cols[:1000])


def test_rmat_quadrant_frequencies(graphs_mod):
    """Before the permutation, the (row bit, column bit) pair at every bit level follows
    (A, B, C, D) = (.57, .19, .19, .05): chi-square with 3 degrees of freedom under 30."""
    scale = 10
    src, dst = graphs_mod.rmat_edges(scale, 64, seed=5, permute=False)
    p = np.array([0.57, 0.19, 0.19, 0.05])
    for bit in range(scale):
        q = ((src >> bit) & 1) * 2 + ((dst >> bit) & 1)
        obs = np.bincount(q, minlength=4)
        exp = p * src.size
        chi2 = float(((obs - exp) ** 2 / exp).sum())
        assert chi2 < 30.0, (bit, obs, chi2)


def test_uniform(graphs_mod):
    src, dst = graphs_mod.uniform_edges(1000, 200000, seed=2)
    assert src.min() >= 0 and src.max() < 1000
    counts = np.bincount(np.concatenate([src, dst]), minlength=1000)
    assert counts.min() > 300 and counts.max() < 500
    _is_clean_symmetric(graphs_mod.from_edges(1000, src, dst))


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 1), (5, 4, 3), (9, 9, 9)])
def test_grid3d(graphs_mod, dims):
    X, Y, Z = dims
    g = graphs_mod.grid3d(X, Y, Z)
    _is_clean_symmetric(g)
    assert g.nnz == 2 * ((X - 1) * Y * Z + X * (Y - 1) * Z + X * Y * (Z - 1))
    ids = np.arange(X * Y * Z)
    x, y, z = ids % X, (ids // X) % Y, ids // (X * Y)
    expect = ((x > 0).astype(int) + (x < X - 1) + (y > 0) + (y < Y - 1) + (z > 0) + (z < Z - 1))
    assert np.array_equal(g.degrees(), expect)


def test_pick_roots(graphs_mod):
    g = graphs_mod.rmat(12, 16, seed=4)
    r = graphs_mod.pick_roots(g, 64, 99)
    assert r.size == 64 and np.unique(r).size == 64
    assert np.all(g.degrees()[r] > 0)
    assert np.array_equal(r, graphs_mod.pick_roots(g, 64, 99))
    small = graphs_mod.from_edges(6, np.array([0, 2], np.int32), np.array([1, 3], np.int32))
    assert sorted(graphs_mod.pick_roots(small, 10, 1).tolist()) == [0, 1, 2, 3]
