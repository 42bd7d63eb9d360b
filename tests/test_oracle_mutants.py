"""The oracle's pins catch plausible mistakes (CPU only): each case plants one mistake in a
copy of the oracle source (a dropped or doubled level increment, a wrong parent, a stack
instead of a queue, a skipped or shifted neighbour, a wrong m_c sum, a checker condition
removed or weakened, a wrong bitmap bit or word in the one-level expansion), compiles it
apart, and requires the oracle tests to fail against it. The unmodified copy must pass."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bfs_oracle.c")

ROW_LOOP = "for (int64_t e = offsets[u]; e < offsets[u + 1]; ++e) {\n            const int32_t v = cols[e];\n            if (level[v] == -1)"
MUTANTS = {
    "level-not-incremented": ("level[v] = level[u] + 1;", "level[v] = level[u];"),
    "level-plus-two": ("level[v] = level[u] + 1;", "level[v] = level[u] + 2;"),
    "parent-is-self": ("pred[v] = u;\n                queue", "pred[v] = v;\n                queue"),
    "root-parent-unset": ("pred[root] = root;", "pred[root] = -1;"),
    "root-level-one": ("level[root] = 0;", "level[root] = 1;"),
    "stack-not-queue": ("const int32_t u = queue[head++];", "const int32_t u = queue[--tail]; if (tail < head) break;"),
    "last-neighbour-dropped": (ROW_LOOP, ROW_LOOP.replace("e < offsets[u + 1]", "e + 1 < offsets[u + 1]")),
    "first-neighbour-dropped": (ROW_LOOP, ROW_LOOP.replace("e = offsets[u];", "e = offsets[u] + 1;")),
    "reached-count-off": ("    free(queue);\n    return tail;", "    free(queue);\n    return tail - 1;"),
    "mc-counts-unreached": ("if (level[v] >= 0) twice", "if (level[v] >= -1) twice"),
    "mc-not-halved": ("return twice / 2;", "return twice;"),
    "mc-degree-plus-one": ("twice += offsets[v + 1] - offsets[v];", "twice += offsets[v + 1] - offsets[v] + 1;"),
    "mc-skips-root": ("if (level[v] >= 0) twice", "if (level[v] > 0) twice"),
    "tree-levels-not-compared": ("if (level[v] != level_ref[v]) {", "if (0) {"),
    "tree-root-not-checked": ("if (level[root] != 0 || pred[root] != root) {", "if (0) {"),
    "tree-unreached-not-paired": ("if ((pred[v] == -1) != (level[v] == -1)) {", "if (0) {"),
    "tree-edge-not-checked": ("if (p < 0 || p >= n || !has_edge(offsets, cols, p, (int32_t)v)) {", "if (p < 0 || p >= n) {"),
    "tree-edge-transposed": ("!has_edge(offsets, cols, p, (int32_t)v)", "!has_edge(offsets, cols, (int32_t)v, (int32_t)v)"),
    "tree-parent-level-weak": ("if (level[p] != level[v] - 1) {", "if (level[p] > level[v]) {"),
    "has-edge-any-larger": ("return lo < offsets[u + 1] && cols[lo] == v;", "return lo < offsets[u + 1];"),
    "has-edge-bound-off": ("if (cols[mid] < v)", "if (cols[mid] <= v)"),
    "edges-gap-two-allowed": ("(a - b > 1 || b - a > 1)", "(a - b > 2 || b - a > 2)"),
    "edges-reach-not-paired": ("if ((a < 0) != (b < 0) || ", "if ("),
    "expand-bit-not-set": ("bitmap[v / 32] |= m;", ";"),
    "expand-parent-is-self": ("pred[v] = u;\n            level[v] = lvl;", "pred[v] = v;\n            level[v] = lvl;"),
    "expand-level-plus-one": ("level[v] = lvl;", "level[v] = lvl + 1;"),
    "expand-wrong-bit": ("const uint32_t m = 1u << (v % 32);", "const uint32_t m = 1u << ((v + 1) % 32);"),
    "expand-wrong-word": ("if (bitmap[v / 32] & m) continue;\n            bitmap[v / 32] |= m;",
                          "if (bitmap[v / 33] & m) continue;\n            bitmap[v / 33] |= m;"),
}


def _run_pins_against(src_text: str, tmp_path, tag: str) -> int:
    c = tmp_path / f"oracle_{tag}.c"
    lib = tmp_path / f"liboracle_{tag}.so"
    c.write_text(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", str(c), "-o", str(lib)], check=True)
    env = dict(os.environ, GBFS_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode


def test_unmodified_copy_passes(tmp_path):
    with open(SRC) as f:
        assert _run_pins_against(f.read(), tmp_path, "unmodified") == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    with open(SRC) as f:
        src = f.read()
    find, repl = MUTANTS[name]
    assert src.count(find) == 1, "the mutated passage no longer appears exactly once in the oracle"
    rc = _run_pins_against(src.replace(find, repl), tmp_path, name)
    assert rc != 0, f"mutant {name} survived the pins"
    assert rc == 1 or rc < 0, f"pytest exit code {rc}: the run did not get as far as the pins"
