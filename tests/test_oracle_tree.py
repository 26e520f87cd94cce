"""Oracle pins for the binary tree (Sec. 2.7, Fig. 1)."""
import numpy as np
import pytest

from conftest import golden_path
from oracle.tree import build_tree


def _read_golden():
    rows, meta = [], {}
    for line in open(golden_path("fig1_tree.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0].isalpha() or "_" in parts[0]:
            meta[parts[0]] = int(parts[1])
        else:
            rows.append(tuple(int(p) for p in parts))
    return meta, rows


def test_fig1_numbering():
    meta, rows = _read_golden()
    t = build_tree(meta["N"], meta["leaf_size"])
    assert t.L == meta["L"]
    for node, first, last in rows:
        assert int(t.start[node]) == first - 1
        assert int(t.start[node] + t.size[node]) == last


@pytest.mark.parametrize("N,m", [(1, 4), (7, 4), (400, 50), (1000, 64), (2112, 64), (4097, 128), (65536, 256)])
def test_partition_and_leaf_size(N, m):
    t = build_tree(N, m)
    for level in range(t.L + 1):
        nodes = list(t.level_nodes(level))
        starts = [int(t.start[x]) for x in nodes]
        ends = [int(t.start[x] + t.size[x]) for x in nodes]
        assert starts[0] == 0 and ends[-1] == N
        assert all(e == s for e, s in zip(ends[:-1], starts[1:]))
    sizes = [int(t.size[x]) for x in t.leaves()]
    assert max(sizes) <= m
    if t.L > 0:
        assert max(int(t.size[x]) for x in t.level_nodes(t.L - 1)) > m
    # children split floor/ceil
    for tau in range(1, 2 ** t.L):
        assert t.size[2 * tau] == t.size[tau] // 2
