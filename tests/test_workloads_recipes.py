"""The seeded input recipes shared by the oracle and the device side, checked
against their stated definitions on the CPU: the batched workload's size and
rank distribution, the exact off-diagonal rank of the synthetic HODLR matrices,
and the tree rule (the same as the method's tree, Sec. 2.7)."""
import numpy as np
import pytest

import workloads as W
from oracle.tree import build_tree


def test_batched_specs_follow_the_recipe():
    specs = W.batched_hodlr_specs(64)
    assert specs == W.batched_hodlr_specs(64)  # seeded
    assert len(specs) == 64
    ns = np.array([s["N"] for s in specs])
    ks = np.array([s["k"] for s in specs])
    assert np.all(ns % 64 == 0) and ns.min() >= 2048 and ns.max() <= 32768
    assert ks.min() >= 8 and ks.max() <= 40
    # log-uniform sizes: the geometric mean sits near sqrt(2048 * 32768) = 8192
    assert 8192 / 1.6 < np.exp(np.mean(np.log(ns))) < 8192 * 1.6
    assert len({s["op_seed"] for s in specs}) == 64
    assert len({s["omega_seed"] for s in specs}) == 64


@pytest.mark.parametrize("N,m,k", [(600, 40, 5), (1000, 64, 9)])
def test_synthetic_hodlr_has_exact_off_diagonal_rank(N, m, k):
    f = W.synthetic_hodlr_factors(N, m, k, seed=7, shift=float(N))
    A = W.dense_from_factors(f)
    L, start, size = f["L"], f["start"], f["size"]
    for j in range(1, L + 1):
        for a in range(2 ** j, 2 ** (j + 1)):
            b = a ^ 1
            blk = A[start[a]:start[a] + size[a], start[b]:start[b] + size[b]]
            assert np.linalg.matrix_rank(blk) == min(k, blk.shape[0], blk.shape[1]), (j, a)
    # leaf blocks: N(0, 1) entries plus the shift on the diagonal
    for i, t in enumerate(range(2 ** L, 2 ** (L + 1))):
        blk = A[start[t]:start[t] + size[t], start[t]:start[t] + size[t]]
        assert np.array_equal(blk, f["D"][i])
        assert abs(np.mean(np.diag(blk)) - N) < 1.0


@pytest.mark.parametrize("N,m", [(1, 4), (7, 3), (1000, 64), (3000, 100), (65536, 256)])
def test_tree_rule_equals_the_oracle_tree(N, m):
    L, start, size = W.tree_ranges(N, m)
    t = build_tree(N, m)
    assert L == t.L
    assert np.array_equal(start, t.start[:len(start)]) and np.array_equal(size, t.size[:len(size)])
