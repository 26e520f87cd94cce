"""Binary index tree (Sec. 2.7, Fig. 1).

The root I_1 = [0, N) is split into two roughly equal halves, recursively,
until every interval holds at most ``leaf_size`` indices.  Heap numbering:
root = 1, children of tau are 2*tau and 2*tau + 1; the nodes on level l are
2**l .. 2**(l+1) - 1.

Reading of the paper (its text allows uneven depth when N / m is not a power
of two, while its algorithms loop over complete levels): every leaf sits on
level L = ceil(log2(N / m)) (L = 0 when N <= m), and a node of size n splits
into floor(n / 2) indices on the left and n - floor(n / 2) on the right.  The
index sets are contiguous; the caller orders the points.

Pinned by tests/test_oracle_tree.py against the numbering printed in Fig. 1
(N = 400 -> 200/200 -> 100 -> 50).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Tree:
    N: int
    leaf_size: int
    L: int
    start: np.ndarray  # int64, indexed by heap id (entry 0 unused)
    size: np.ndarray   # int64, indexed by heap id

    def level_nodes(self, level: int) -> range:
        return range(2 ** level, 2 ** (level + 1))

    def leaves(self) -> range:
        return self.level_nodes(self.L)

    def rows(self, node: int) -> slice:
        s = int(self.start[node])
        return slice(s, s + int(self.size[node]))

    @property
    def n_max(self) -> int:
        return int(max(self.size[t] for t in self.leaves()))


def num_levels(N: int, leaf_size: int) -> int:
    if N <= leaf_size:
        return 0
    return int(math.ceil(math.log2(N / leaf_size) - 1e-12))


def build_tree(N: int, leaf_size: int) -> Tree:
    """Uniform-depth binary tree over [0, N) with leaves of at most leaf_size."""
    if N < 1 or leaf_size < 1:
        raise ValueError("N and leaf_size must be positive")
    L = num_levels(N, leaf_size)
    # guard against floating-point in the log: smallest L with ceil(N / 2^L) <= m
    while L > 0 and -(-N // 2 ** (L - 1)) <= leaf_size:
        L -= 1
    while -(-N // 2 ** L) > leaf_size:
        L += 1
    nnodes = 2 ** (L + 1)
    start = np.zeros(nnodes, dtype=np.int64)
    size = np.zeros(nnodes, dtype=np.int64)
    start[1], size[1] = 0, N
    for tau in range(1, 2 ** L):
        n = int(size[tau])
        left = n // 2
        start[2 * tau], size[2 * tau] = start[tau], left
        start[2 * tau + 1], size[2 * tau + 1] = start[tau] + left, n - left
    return Tree(N=N, leaf_size=leaf_size, L=L, start=start, size=size)
