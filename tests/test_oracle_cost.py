"""Cost-scaling pins of the oracle (Sec. 3.1 HODLR complexity, Sec. 4.4 HBS
complexity, Sec. 5 tables: T_net and the storage M).

T_net (the compression's own arithmetic, black box excluded) is counted in
floating-point operations by ``oracle.cost``.  With N = m 2^L and every node of
a level the same size, the count divided by N is a polynomial in the number of
levels L = log2(N / m):
  HODLR: the peel at level l applies l levels of factors, so T_net / N is
         quadratic in L (O(k^2 N log^2 N));
  HBS:   the nested partial apply touches one level of long bases, so T_net / N
         is linear in L (O(k^2 N log N)), up to terms that vanish as 1/N.
The stored reals per point, M / N, grow linearly in L for HODLR (one pair of
N x k bases per level) and stay flat for HBS (one pair of leaf bases).
"""
import numpy as np

import workloads as W
from oracle import cost
from oracle import grad as ograd
from oracle import hbs as ohbs
from oracle import hodlr as ohodlr
from oracle.tree import build_tree

M_LEAF, K, P = 32, 6, 6
LEVELS = [4, 5, 6, 7, 8]


def _black_box(N):
    f = W.synthetic_hodlr_factors(N, M_LEAF, K, seed=9, shift=float(N))
    return lambda X, transpose: ograd.apply(f, X, transpose)


def _counts(kind):
    g, mem = [], []
    for L in LEVELS:
        N = M_LEAF * 2 ** L
        t = build_tree(N, M_LEAF)
        assert t.L == L
        cost.reset()
        if kind == "hodlr":
            h = ohodlr.compress(_black_box(N), t, r=K + P, k=K, seed=2)
            stored = sum(h.U[a].size + h.V[a].size + np.count_nonzero(np.diag(h.B[a]))
                         for a in range(2, 2 ** (L + 1))) + sum(d.size for d in h.D.values())
        else:
            h = ohbs.compress(_black_box(N), t, r=K + P, seed=2)
            leaves = list(t.leaves())
            stored = (sum(h.Ulong[x].size + h.Vlong[x].size for x in leaves)
                      + sum(h.Ushort[x].size + h.Vshort[x].size for x in h.Ushort)
                      + sum(b.size for b in h.B.values()) + sum(d.size for d in h.D.values()))
        g.append(cost.COUNT.flops / N)
        mem.append(stored / N)
    return np.array(g), np.array(mem)


def test_hodlr_net_cost_is_k2_n_log2_n():
    g, mem = _counts("hodlr")
    d1, d2, d3 = np.diff(g), np.diff(g, 2), np.diff(g, 3)
    # quadratic in L: positive second difference, constant up to terms of
    # order 1 / N (the third difference is a tiny fraction of it)
    assert np.all(d2 > 0.05 * d1[:-1])
    assert np.max(np.abs(d3)) <= 0.02 * np.min(d2)
    assert d2.max() / d2.min() < 1.05
    # the L^2 term leads: T_net / (N L^2) stays within +-30% over the range while
    # T_net / (N L) keeps growing
    lead = g / np.array(LEVELS, float) ** 2
    assert lead.max() / lead.min() < 1.3 ** 2
    per_level = g / np.array(LEVELS, float)
    assert np.all(np.diff(per_level) > 0)
    # storage: one pair of N x k bases per level -> M / N = 2 k L + const (the k
    # diagonal entries of B per node add 2^(L+1) k / N, which vanishes as 1 / m)
    assert np.allclose(np.diff(mem), 2 * K, rtol=0, atol=2.0 * K / M_LEAF)


def test_hbs_net_cost_is_k2_n_log_n():
    g, mem = _counts("hbs")
    d1, d2 = np.diff(g), np.diff(g, 2)
    # linear in L up to corrections that die out geometrically with L (the
    # root level's narrower panels, node counts 2^l - 1 instead of 2^l): the
    # growth per added level converges, the second difference halves per level
    assert np.all(d1 > 0)
    assert abs(d1[-1] - d1[-2]) <= 0.05 * d1[-1]
    assert np.all(np.abs(d2[1:]) <= 0.6 * np.abs(d2[:-1]))
    lead = g / np.array(LEVELS, float)
    assert lead.max() / lead.min() < 1.3 ** 2
    # storage per point is flat: leaf bases, short bases, sibling and leaf blocks
    assert mem.max() / mem.min() < 1.05


def test_hodlr_and_hbs_costs_separate():
    """The counts tell the two laws apart over the same range: the HODLR growth
    per added level increases, the HBS growth per added level does not."""
    gh, _ = _counts("hodlr")
    gb, _ = _counts("hbs")
    assert np.diff(gh)[-1] / np.diff(gh)[0] > 1.3
    assert np.diff(gb)[-1] / np.diff(gb)[0] < 1.0
