"""HODLR compression by randomized peeling (Sec. 3, Fig. "Randomized compression
of a HODLR matrix"), with the level-truncated apply A^(l) of Sec. 2.8.

Format (Sec. 2.8 with Remark 4, diagonal sibling matrices): for every sibling
pair {alpha, beta} below the root, A(I_alpha, I_beta) ~= U_alpha B_alphabeta
V_beta^T with orthonormal long bases, and a dense D_tau for every leaf.
``U[a]`` / ``B[a]`` / ``V[a ^ 1]`` hold the factors of the block (a, sibling);
the rank of that block is the column count of U[a].

Readings of the paper:
* The factorization display of Sec. 2.8 is read as A_ab = U_a B_ab V_b^T with
  U, V orthonormal.
* In the figure the second SVD of a sibling pair returns \\hat U_alpha (the
  figure prints \\hat V_alpha); derivation: Z2(I_beta,:) = A_ab^T U_a.
* Test matrix packing: X = [Omega_2 | Omega_1] so that columns 0..r-1 of
  A X are Y_1 and columns r..2r-1 are Y_2; Omega_2 is nonzero on right
  children, Omega_1 on left children (both from one Gaussian field per level).
* Tolerance mode: the paper's eps is absolute (Sec. 2.6 mode 3); a relative
  ``tol`` is turned into eps = tol * nu, nu = the largest singular value met in
  the two level-0 SVDs (a lower bound for ||A||_2 known after the first A^T
  step), kept fixed for the run.  With eps = tol * nu the relative Frobenius
  error of the log-kernel workloads came out at 1.4e-7-1.6e-7 (> tol), so the
  threshold is eps = EPS_SCALE * tol * nu with EPS_SCALE = 0.1.  Fixed-rank
  mode keeps exactly k terms.

Pinned by tests/test_oracle_hodlr.py: exact recovery of a seeded HODLR matrix
of rank k <= r to rounding, detected ranks equal to brute-force dense SVD
ranks, the randomized range-finder bound (Sec. 2.5), matvec column counts
linear in the number of levels, and dense A^(l) against blockwise masking.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import numpy as np

from .cost import mm, svd
from .lowrank import qr_basis, range_basis, svd_trunc
from .philox import level_field
from .tree import Tree

EPS_SCALE = 0.1

ApplyFn = Callable[[np.ndarray, bool], np.ndarray]  # (X, transpose) -> op(A) @ X


@dataclass
class HODLR:
    tree: Tree
    U: dict = field(default_factory=dict)
    V: dict = field(default_factory=dict)
    B: dict = field(default_factory=dict)
    D: dict = field(default_factory=dict)
    cols_A: int = 0
    cols_At: int = 0
    eps_abs: float | None = None

    def rank(self, a: int) -> int:
        return int(self.U[a].shape[1])


def partial_apply(h: HODLR, level: int, X: np.ndarray, transpose: bool = False) -> np.ndarray:
    """A^(level) X (or its transpose): sum of the compressed sibling blocks of
    node levels 1..level (Sec. 2.8), evaluated block by block."""
    t = h.tree
    Y = np.zeros_like(X, dtype=np.float64)
    for j in range(1, level + 1):
        for a in t.level_nodes(j):
            b = a ^ 1
            Ia, Ib = t.rows(a), t.rows(b)
            if not transpose:
                Y[Ia] += mm(h.U[a], mm(h.B[a], mm(h.V[b].T, X[Ib])))
            else:
                Y[Ib] += mm(h.V[b], mm(h.B[a].T, mm(h.U[a].T, X[Ia])))
    return Y


def apply(h: HODLR, X: np.ndarray, transpose: bool = False) -> np.ndarray:
    """Full compressed apply: block-diagonal D plus A^(L)."""
    t = h.tree
    Y = partial_apply(h, t.L, X, transpose)
    for tau in t.leaves():
        I = t.rows(tau)
        Y[I] += mm(h.D[tau].T if transpose else h.D[tau], X[I])
    return Y


def dense(h: HODLR) -> np.ndarray:
    return apply(h, np.eye(h.tree.N))


def gaussian_test_matrix(tree: Tree, level: int, r: int, seed: int, mixed: bool) -> np.ndarray:
    """X = [Omega_2 | Omega_1] for the parents on ``level``: Omega_1 = G on the
    left child of every parent, Omega_2 = G on the right child."""
    G = level_field(seed, level, tree.N, r, mixed)
    X = np.zeros((tree.N, 2 * r))
    for tau in tree.level_nodes(level):
        a, b = 2 * tau, 2 * tau + 1
        X[tree.rows(b), :r] = G[tree.rows(b)]
        X[tree.rows(a), r:] = G[tree.rows(a)]
    return X


def identity_test_matrix(tree: Tree) -> np.ndarray:
    """Omega(I_tau, 1:n_tau) = I for every leaf, zero padded to n_max columns."""
    X = np.zeros((tree.N, tree.n_max))
    for tau in tree.leaves():
        n = int(tree.size[tau])
        X[tree.rows(tau), :n] = np.eye(n)
    return X


def compress(apply_A: ApplyFn, tree: Tree, r: int, k: int | None = None,
             tol: float | None = None, seed: int = 2, mixed: bool = False,
             basis: str = "qr") -> HODLR:
    """Fig. "Randomized compression of a HODLR matrix", level by level.

    basis: how U_alpha = qr(Y1(I_alpha,:)) is read: "qr" is the Q factor of a
    full Householder QR (r columns); "range" keeps only the numerical range
    (``range_basis``).  The two agree on the range of the samples and differ in
    the directions that are rounding noise, which pick up the coarser levels'
    truncation error through the transpose peel.
    """
    orth = qr_basis if basis == "qr" else range_basis
    if (k is None) == (tol is None):
        raise ValueError("exactly one of k (fixed rank) or tol (adaptive) is required")
    h = HODLR(tree=tree)
    for level in range(tree.L):
        # random test matrices and the samples for the incoming bases
        X = gaussian_test_matrix(tree, level, r, seed, mixed)
        Y = apply_A(X, False) - partial_apply(h, level, X)
        h.cols_A += X.shape[1]
        # orthonormalize: U_alpha = qr(Y1(I_alpha,:)), U_beta = qr(Y2(I_beta,:))
        Xt = np.zeros_like(X)
        Ucur = {}
        for tau in tree.level_nodes(level):
            a, b = 2 * tau, 2 * tau + 1
            Ucur[a] = orth(Y[tree.rows(a), :r])
            Ucur[b] = orth(Y[tree.rows(b), r:])
            # Omega_1(I_alpha,:) = U_alpha, Omega_2(I_beta,:) = U_beta (a node with
            # fewer than r rows has a square basis; the remaining columns stay zero)
            Xt[tree.rows(a), r:r + Ucur[a].shape[1]] = Ucur[a]
            Xt[tree.rows(b), :Ucur[b].shape[1]] = Ucur[b]
        # samples for the outgoing bases
        Z = apply_A(Xt, True) - partial_apply(h, level, Xt, transpose=True)
        h.cols_At += Xt.shape[1]
        svds = {}
        for tau in tree.level_nodes(level):
            a, b = 2 * tau, 2 * tau + 1
            svds[tau] = (svd(Z[tree.rows(a), :r]),  # A_ba^T U_b
                         svd(Z[tree.rows(b), r:]))  # A_ab^T U_a
        if tol is not None and h.eps_abs is None:
            h.eps_abs = EPS_SCALE * tol * max(max(s1[1][0], s2[1][0]) for s1, s2 in svds.values())
        for tau in tree.level_nodes(level):
            a, b = 2 * tau, 2 * tau + 1
            (Va, sa, Wat), (Vb, sb, Wbt) = svds[tau]
            # [V_a, B_ba, \hat U_b] = svd(Z1(I_a,:)); [V_b, B_ab, \hat U_a] = svd(Z2(I_b,:))
            Va, sa, Wat = _truncate(Va, sa, Wat, k, h.eps_abs)
            Vb, sb, Wbt = _truncate(Vb, sb, Wbt, k, h.eps_abs)
            h.V[a], h.B[b], h.U[b] = Va, np.diag(sa), mm(Ucur[b], Wat[:, :Ucur[b].shape[1]].T)
            h.V[b], h.B[a], h.U[a] = Vb, np.diag(sb), mm(Ucur[a], Wbt[:, :Ucur[a].shape[1]].T)
    # diagonal blocks: Y = A Omega - A^(L) Omega with the identity probe
    X = identity_test_matrix(tree)
    Y = apply_A(X, False) - partial_apply(h, tree.L, X)
    h.cols_A += X.shape[1]
    for tau in tree.leaves():
        n = int(tree.size[tau])
        h.D[tau] = Y[tree.rows(tau), :n].copy()
    return h


def _truncate(U, s, Vt, k, eps):
    n = s.size
    if k is not None:
        n = min(n, int(k))
    if eps is not None:
        n = min(n, max(1, int(np.count_nonzero(s > eps))))
    return U[:, :n], s[:n], Vt[:n]


def dense_apply_fn(A: np.ndarray) -> ApplyFn:
    """Black box for a dense operator held in memory (applied in FP64)."""
    A64 = np.asarray(A, dtype=np.float64)

    def f(X, transpose):
        return (A64.T @ X) if transpose else (A64 @ X)
    return f


__all__ = ["HODLR", "compress", "partial_apply", "apply", "dense", "gaussian_test_matrix",
           "identity_test_matrix", "dense_apply_fn", "svd_trunc"]
