"""Text edge lists (the format of the SNAP graphs in the paper's Table 3, Sec. 5): the
parser against a plain line-by-line reading, file order kept across thread splits, errors
naming the first bad line, gzip files, id compaction, and the built CSR (CPU only)."""
import gzip

import numpy as np
import pytest


def _plain_parse(text: str):
    """Line-by-line statement of the format: blank and '#'/'%' lines skipped, the first two
    fields of every other line are the pair (separators: blanks, tabs, commas)."""
    src, dst = [], []
    for line in text.split("\n"):
        s = line.strip(" \t\r\v\f")
        if not s or s[0] in "#%":
            continue
        fields = s.replace(",", " ").split()
        src.append(int(fields[0]))
        dst.append(int(fields[1]))
    return np.array(src, np.int64), np.array(dst, np.int64)


def _random_text(rng, lines: int) -> str:
    out = []
    for i in range(lines):
        k = rng.integers(0, 20)
        if k == 0:
            out.append("# comment " + "x" * int(rng.integers(0, 40)))
        elif k == 1:
            out.append(" " * int(rng.integers(0, 3)))
        elif k == 2:
            out.append("% other comment")
        else:
            u, v = (int(x) for x in rng.integers(0, 1 << int(rng.integers(1, 31)), 2))
            sep = [" ", "\t", ",", ", ", "  \t"][int(rng.integers(0, 5))]
            tail = ["", "\t1", " 3.25", "\r", " 17 18\r"][int(rng.integers(0, 5))]
            lead = ["", " ", "\t"][int(rng.integers(0, 3))]
            out.append(f"{lead}{u}{sep}{v}{tail}")
    return "\n".join(out) + ("\n" if rng.integers(0, 2) else "")


@pytest.mark.parametrize("threads", [1, 3, 8, 16])
def test_parse_matches_plain_reading(graphs_mod, threads):
    rng = np.random.default_rng(threads)
    text = _random_text(rng, 60000)  # > 1 MB: split into pieces at line starts
    src, dst, max_id = graphs_mod.parse_edge_list(text.encode(), threads=threads)
    ps, pd = _plain_parse(text)
    assert np.array_equal(src, ps) and np.array_equal(dst, pd)  # file order kept
    assert max_id == max(ps.max(), pd.max())


def test_parse_edge_cases(graphs_mod):
    src, dst, max_id = graphs_mod.parse_edge_list(b"")
    assert src.size == 0 and max_id == -1
    src, dst, max_id = graphs_mod.parse_edge_list(b"# only a comment\n\n")
    assert src.size == 0 and max_id == -1
    src, dst, max_id = graphs_mod.parse_edge_list(b"0 2147483646")  # no final newline, largest id
    assert src.tolist() == [0] and dst.tolist() == [2147483646] and max_id == 2147483646


@pytest.mark.parametrize("bad,line,what", [
    (b"1 2\n3\n", 2, "not a pair"), (b"1 2\n4 -5\n", 2, "not a pair"), (b"x y\n", 1, "not a pair"),
    (b"1 2x\n", 1, "not a pair"), (b"1 2\n# c\n\n2147483647 0\n", 4, "above"),
    (b"7 99999999999999999999999\n", 1, "above")])
def test_parse_errors_name_the_line(graphs_mod, bad, line, what):
    with pytest.raises(ValueError, match=f"line {line}: .*{what}"):
        graphs_mod.parse_edge_list(bad)


def test_parse_error_late_in_a_large_file(graphs_mod):
    rng = np.random.default_rng(4)
    lines = [f"{a} {b}" for a, b in rng.integers(0, 1000, (80000, 2))]
    lines[70001] = "12 oops"
    with pytest.raises(ValueError, match="line 70002:"):
        graphs_mod.parse_edge_list(("\n".join(lines) + "\n").encode(), threads=8)


def test_load_file_gzip_and_compaction(graphs_mod, tmp_path):
    text = "# a 5-cycle with file ids 10, 20, ..., 50, a repeated edge and a loop\n" \
           "10 20\n20 30\n30 40\n40 50\n50 10\n20 10\n30 30\n"
    plain, gz = tmp_path / "c.txt", tmp_path / "c.txt.gz"
    plain.write_text(text)
    with gzip.open(gz, "wt") as f:
        f.write(text)
    for path in (plain, gz):
        g = graphs_mod.load_edge_list(str(path))
        assert g.n == 51 and g.nnz == 10 and g.ids is None
        assert g.degrees()[10::10].tolist() == [2] * 5 and g.degrees().sum() == 10
        c = graphs_mod.load_edge_list(str(path), compact=True)
        assert c.n == 5 and c.ids.tolist() == [10, 20, 30, 40, 50]
        assert np.array_equal(c.offsets, np.arange(0, 11, 2))
        assert c.cols.tolist() == [1, 4, 0, 2, 1, 3, 2, 4, 0, 3]
    (tmp_path / "empty.txt").write_text("")
    with pytest.raises(ValueError, match="no edges"):
        graphs_mod.load_edge_list(str(tmp_path / "empty.txt"))
    (tmp_path / "bad.txt").write_text("1 2\n3 4 \n5\n")
    with pytest.raises(ValueError, match="bad.txt: edge list line 3"):
        graphs_mod.load_edge_list(str(tmp_path / "bad.txt"))


def test_loaded_graph_equals_generated(graphs_mod, oracle_mod, tmp_path):
    """An R-MAT edge list written out and read back builds the same CSR as the generator,
    and the oracle gives the same levels on it."""
    src, dst = graphs_mod.rmat_edges(12, 8, seed=9)
    path = tmp_path / "rmat.txt"
    np.savetxt(path, np.stack([src, dst], 1), fmt="%d", delimiter="\t", header="R-MAT s12 ef8", comments="# ")
    g = graphs_mod.load_edge_list(str(path))
    ref = graphs_mod.from_edges(int(max(src.max(), dst.max())) + 1, src, dst)
    assert np.array_equal(g.offsets, ref.offsets) and np.array_equal(g.cols, ref.cols)
    root = int(graphs_mod.pick_roots(g, 1, 5)[0])
    assert np.array_equal(oracle_mod.bfs(g.offsets, g.cols, root)[0], oracle_mod.bfs(ref.offsets, ref.cols, root)[0])


MTX = """%%MatrixMarket matrix coordinate real symmetric
% a 4-cycle 1-2-3-4-1 plus a pendant vertex 6 on 4; vertex 5 is isolated
%
6 6 6
2 1 1.5
3 2 -2e3
4 3 7
4 1 0.25
6 4 1
4 4 3.0
"""


def test_matrix_market(graphs_mod, oracle_mod, tmp_path):
    plain, gz = tmp_path / "g.mtx", tmp_path / "g.mtx.gz"
    plain.write_text(MTX)
    with gzip.open(gz, "wt") as f:
        f.write(MTX)
    for path in (plain, gz):
        g = graphs_mod.load_edge_list(str(path))
        assert g.n == 6 and g.nnz == 10  # the diagonal entry (4, 4) is a loop: removed
        assert g.degrees().tolist() == [2, 2, 2, 3, 0, 1]
        lv, _ = oracle_mod.bfs(g.offsets, g.cols, 0)
        assert lv.tolist() == [0, 1, 2, 1, -1, 2]
        c = graphs_mod.load_edge_list(str(path), compact=True)
        assert c.n == 5 and c.ids.tolist() == [0, 1, 2, 3, 5]


@pytest.mark.parametrize("text,match", [
    ("%%MatrixMarket matrix array real general\n2 2\n1\n2\n3\n4\n", "only 'matrix coordinate'"),
    ("%%MatrixMarket matrix coordinate pattern general\n% c\n", "no size line"),
    ("%%MatrixMarket matrix coordinate pattern general\n% c\n3 3\n1 2\n", "line 3: expected"),
    ("%%MatrixMarket matrix coordinate pattern general\n3 3 2\n1 2\n", "1 entries, the size line says 2"),
    ("%%MatrixMarket matrix coordinate pattern general\n3 3 2\n1 2\n0 3\n", "outside"),
    ("%%MatrixMarket matrix coordinate pattern general\n3 3 2\n1 2\n2 4\n", "outside"),
    ("%%MatrixMarket matrix coordinate pattern general\n%\n3 3 2\n1 2\n2 x\n", "line 5: not a pair")])
def test_matrix_market_errors(graphs_mod, tmp_path, text, match):
    path = tmp_path / "bad.mtx"
    path.write_text(text)
    with pytest.raises(ValueError, match=match):
        graphs_mod.load_edge_list(str(path))
