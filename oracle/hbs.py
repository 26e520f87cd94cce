"""HBS compression (Sec. 4.1, Fig. "A basic scheme for compressing an HBS
matrix"), the partial apply A^(m) (Fig. "Application of A^(m) in the HBS
framework") and the conversion to HBS-ID with adaptive ranks (Sec. 4.3,
Fig. "An algorithm for computing the HBS-ID representation").

The oracle keeps every long basis explicitly (the basic scheme); the storage
efficient scheme of Sec. 4.2 computes the same numbers and keeps only the
current level's long bases plus the vectors y, z.

Readings of the paper:
* Sibling matrices: the figure assigns X1 to B_alphabeta; from
  Z1^loc(:, 1:r) = A_ba^T U_b = V_a diag(b21) X1(1:r,:)^T it follows that
  B_ba = X1(1:r,:) diag(b21) and B_ab = X2(1:r,:) diag(b12).
* The downward pass of the partial-apply figure is printed with the upward
  loop bounds; it runs over levels 1 .. m-1 (coarse to fine), and
  U_tau(J_alpha,:) is the alpha half (first r rows for the left child) of the
  short 2r x r matrix.  The transpose swaps U <-> V and B_ab -> B_ba^T.
* HBS-ID: id(Y_tmp^*, eps) gives Y_tmp^T ~= Y_tmp^T(:, J) T, hence
  Y_tmp ~= T^T Y_tmp(J,:); the interpolation matrix of a node is T^T
  (n_tau x k at a leaf, (k_a + k_b) x k at a parent).  The apply of the HBS-ID
  form is the partial-apply figure with these interpolation matrices, the
  skeleton sibling matrices B_skel and the leaf blocks D_tau.
* The ID tolerance is absolute in the paper; a relative tol is turned into
  one threshold per side: eps_in = EPS_SCALE * tol * max(y on level 1) for the
  row skeletons and eps_out = EPS_SCALE * tol * max(z on level 1) for the
  column skeletons (y carries the scale of Gaussian samples, z that of
  orthonormal probes; each side keeps its scale on every level).  The ID
  amplifies the truncation error (the paper's HBS-ID tables show E about ten
  times eps), the FP32 log-kernel operator carries full-rank rounding noise
  of about 3e-8 relative in Frobenius norm, and the rank-r HBS stage leaves
  its own error (about 9e-8 at N = 65536, r = 60); EPS_SCALE = 0.004 keeps the
  relative Frobenius error of the log-kernel workloads below tol = 1e-7 up to
  N = 65536 with a margin that rounding-level changes of the arithmetic do not
  use up (0.01 gave 1.24e-7 there; 0.005 gave 9.5e-8 to 1.0e-7 depending on
  the rounding of the products).

Pinned by tests/test_oracle_hbs.py: exact recovery of a seeded HBS-type matrix,
nestedness U_tau = diag(U_a, U_b) U_tau(short), the long basis spanning the
neutered row block (checked densely), B_skel = A(skeleton rows, skeleton
columns) (Sec. 4.3), HBS-ID error at tol, the partial apply against a dense
masked matrix.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .cost import mm, svd
from .hodlr import ApplyFn, gaussian_test_matrix, identity_test_matrix
from .lowrank import RANGE_FLOOR, fix_signs, interp_decomp
from .tree import Tree

EPS_SCALE = 0.004


@dataclass
class HBS:
    tree: Tree
    r: int
    Ulong: dict = field(default_factory=dict)   # node -> n_node x r
    Vlong: dict = field(default_factory=dict)
    Ushort: dict = field(default_factory=dict)  # non-leaf, non-root node -> 2r x r
    Vshort: dict = field(default_factory=dict)
    B: dict = field(default_factory=dict)       # node a -> B_{a, sibling(a)} (r x r)
    y: dict = field(default_factory=dict)       # node -> r
    z: dict = field(default_factory=dict)
    D: dict = field(default_factory=dict)
    cols_A: int = 0
    cols_At: int = 0


def partial_apply(h: HBS, m: int, Q: np.ndarray, transpose: bool = False) -> np.ndarray:
    """u = A^(m) q (or (A^(m))^T q), following the partial-apply figure.

    Uses the long bases of level m, the short bases of levels 1..m-1 and the
    sibling matrices of levels 1..m.  Q may hold several columns.
    """
    t = h.tree
    out = np.zeros_like(Q, dtype=np.float64)
    if m == 0:
        return out
    Uin, Vout = (h.Vlong, h.Ulong) if transpose else (h.Ulong, h.Vlong)
    Sin, Sout = (h.Vshort, h.Ushort) if transpose else (h.Ushort, h.Vshort)

    def Bmat(a):
        return h.B[a ^ 1].T if transpose else h.B[a]

    qhat = {}
    # outgoing expansions on level m
    for tau in t.level_nodes(m):
        qhat[tau] = mm(Vout[tau].T, Q[t.rows(tau)])
    # upward pass, levels m-1 .. 1
    for lev in range(m - 1, 0, -1):
        for tau in t.level_nodes(lev):
            a, b = 2 * tau, 2 * tau + 1
            qhat[tau] = mm(Sout[tau].T, np.vstack([qhat[a], qhat[b]]))
    # incoming expansions for the children of the root
    uhat = {2: mm(Bmat(2), qhat[3]), 3: mm(Bmat(3), qhat[2])}
    # downward pass, levels 1 .. m-1
    r = h.r
    for lev in range(1, m):
        for tau in t.level_nodes(lev):
            a, b = 2 * tau, 2 * tau + 1
            uhat[a] = mm(Bmat(a), qhat[b]) + mm(Sin[tau][:r], uhat[tau])
            uhat[b] = mm(Bmat(b), qhat[a]) + mm(Sin[tau][r:], uhat[tau])
    # incoming expansions on level m
    for tau in t.level_nodes(m):
        out[t.rows(tau)] = mm(Uin[tau], uhat[tau])
    return out


def apply(h: HBS, X: np.ndarray, transpose: bool = False) -> np.ndarray:
    t = h.tree
    Y = partial_apply(h, t.L, X, transpose)
    for tau in t.leaves():
        I = t.rows(tau)
        Y[I] += mm(h.D[tau].T if transpose else h.D[tau], X[I])
    return Y


def dense(h: HBS) -> np.ndarray:
    return apply(h, np.eye(h.tree.N))


def _svd_r(M: np.ndarray, r: int, floor: bool = False):
    """svd(M, r): the leading r singular triplets.  With floor, directions whose
    singular value is below RANGE_FLOOR * sigma_1 are returned as zero columns
    (significant-range reading, as for ``lowrank.range_basis``)."""
    U, s, Vt = svd(M)
    U, Vt = fix_signs(U, Vt)
    U, s, V = U[:, :r].copy(), s[:r].copy(), Vt[:r].T.copy()
    if floor and s.size:
        dead = ~(s > RANGE_FLOOR * s[0])
        U[:, dead] = 0.0
        V[:, dead] = 0.0
        s[dead] = 0.0
    return U, s, V


def compress(apply_A: ApplyFn, tree: Tree, r: int, seed: int = 2, mixed: bool = False,
             floor: bool = False) -> HBS:
    """Fig. "A basic scheme for compressing an HBS matrix" (fixed rank r).

    floor: read svd(., r) on the numerical range (see ``_svd_r``)."""
    h = HBS(tree=tree, r=r)
    t = tree
    if min(int(t.size[x]) for x in t.leaves()) < r:
        raise ValueError("HBS compression needs every leaf to hold at least r indices")
    for level in range(t.L):
        X = gaussian_test_matrix(t, level, r, seed, mixed)
        Y = apply_A(X, False) - partial_apply(h, level, X)
        h.cols_A += X.shape[1]
        Xt = np.zeros_like(X)
        for tau in t.level_nodes(level):
            a, b = 2 * tau, 2 * tau + 1
            Ja = slice(0, int(t.size[a]))
            Jb = slice(int(t.size[a]), int(t.size[tau]))
            if tau == 1:
                Yloc_a, Yloc_b = Y[t.rows(a), :r], Y[t.rows(b), r:]
            else:
                Ybold = h.Ulong[tau] * h.y[tau][None, :]
                Yloc_a = np.hstack([Y[t.rows(a), :r], Ybold[Ja]])
                Yloc_b = np.hstack([Y[t.rows(b), r:], Ybold[Jb]])
            h.Ulong[a], h.y[a], _ = _svd_r(Yloc_a, r, floor)
            h.Ulong[b], h.y[b], _ = _svd_r(Yloc_b, r, floor)
            Xt[t.rows(a), r:] = h.Ulong[a]
            Xt[t.rows(b), :r] = h.Ulong[b]
            if tau != 1:
                h.Ushort[tau] = np.vstack([mm(h.Ulong[a].T, h.Ulong[tau][Ja]),
                                           mm(h.Ulong[b].T, h.Ulong[tau][Jb])])
        Z = apply_A(Xt, True) - partial_apply(h, level, Xt, transpose=True)
        h.cols_At += Xt.shape[1]
        for tau in t.level_nodes(level):
            a, b = 2 * tau, 2 * tau + 1
            Ja = slice(0, int(t.size[a]))
            Jb = slice(int(t.size[a]), int(t.size[tau]))
            if tau == 1:
                Zloc_a, Zloc_b = Z[t.rows(a), :r], Z[t.rows(b), r:]
            else:
                Zbold = h.Vlong[tau] * h.z[tau][None, :]
                Zloc_a = np.hstack([Z[t.rows(a), :r], Zbold[Ja]])
                Zloc_b = np.hstack([Z[t.rows(b), r:], Zbold[Jb]])
            h.Vlong[a], b21, X1 = _svd_r(Zloc_a, r, floor)
            h.Vlong[b], b12, X2 = _svd_r(Zloc_b, r, floor)
            h.z[a], h.z[b] = b21, b12
            h.B[b] = X1[:r] * b21[None, :]   # B_ba = X1(1:r,:) diag(b21)
            h.B[a] = X2[:r] * b12[None, :]   # B_ab = X2(1:r,:) diag(b12)
            if tau != 1:
                h.Vshort[tau] = np.vstack([mm(h.Vlong[a].T, h.Vlong[tau][Ja]),
                                           mm(h.Vlong[b].T, h.Vlong[tau][Jb])])
    X = identity_test_matrix(t)
    Y = apply_A(X, False) - partial_apply(h, t.L, X)
    h.cols_A += X.shape[1]
    for tau in t.leaves():
        n = int(t.size[tau])
        h.D[tau] = Y[t.rows(tau), :n].copy()
    return h


# ---------------------------------------------------------------- HBS-ID ----

@dataclass
class HBSID:
    tree: Tree
    Tin: dict = field(default_factory=dict)    # node -> k_in x (n_leaf or k_a + k_b)
    Tout: dict = field(default_factory=dict)
    Iin: dict = field(default_factory=dict)    # node -> global skeleton row indices
    Iout: dict = field(default_factory=dict)   # node -> global skeleton column indices
    Bskel: dict = field(default_factory=dict)  # node a -> k_in(a) x k_out(sibling)
    D: dict = field(default_factory=dict)
    eps_in: float = 0.0
    eps_out: float = 0.0

    def rank_in(self, tau):
        return int(self.Tin[tau].shape[0])

    def rank_out(self, tau):
        return int(self.Tout[tau].shape[0])


def to_hbsid(h: HBS, tol: float | None = None, k: int | None = None) -> HBSID:
    """Fig. "An algorithm for computing the HBS-ID representation": upward sweep."""
    t = h.tree
    out = HBSID(tree=t)
    eps_in = eps_out = None
    if tol is not None:
        eps_in = EPS_SCALE * tol * max(float(np.max(h.y[2])), float(np.max(h.y[3])))
        eps_out = EPS_SCALE * tol * max(float(np.max(h.z[2])), float(np.max(h.z[3])))
        out.eps_in, out.eps_out = eps_in, eps_out
    Usamp, Vsamp = {}, {}
    for tau in t.leaves():
        Ytmp = h.Ulong[tau] * h.y[tau][None, :]
        Ztmp = h.Vlong[tau] * h.z[tau][None, :]
        Jin, Tin = interp_decomp(Ytmp.T, k=k, eps=eps_in)
        Jout, Tout = interp_decomp(Ztmp.T, k=k, eps=eps_out)
        out.Tin[tau], out.Tout[tau] = Tin, Tout
        out.Iin[tau] = int(t.start[tau]) + Jin
        out.Iout[tau] = int(t.start[tau]) + Jout
        Usamp[tau] = h.Ulong[tau][Jin]
        Vsamp[tau] = h.Vlong[tau][Jout]
    for lev in range(t.L - 1, 0, -1):
        for tau in t.level_nodes(lev):
            a, b = 2 * tau, 2 * tau + 1
            Utmp = _blkdiag(Usamp[a], Usamp[b]) @ h.Ushort[tau]
            Vtmp = _blkdiag(Vsamp[a], Vsamp[b]) @ h.Vshort[tau]
            Jin, Tin = interp_decomp((Utmp * h.y[tau][None, :]).T, k=k, eps=eps_in)
            Jout, Tout = interp_decomp((Vtmp * h.z[tau][None, :]).T, k=k, eps=eps_out)
            out.Tin[tau], out.Tout[tau] = Tin, Tout
            out.Iin[tau] = np.concatenate([out.Iin[a], out.Iin[b]])[Jin]
            out.Iout[tau] = np.concatenate([out.Iout[a], out.Iout[b]])[Jout]
            Usamp[tau], Vsamp[tau] = Utmp[Jin], Vtmp[Jout]
            out.Bskel[a] = Usamp[a] @ h.B[a] @ Vsamp[b].T
            out.Bskel[b] = Usamp[b] @ h.B[b] @ Vsamp[a].T
    out.Bskel[2] = Usamp[2] @ h.B[2] @ Vsamp[3].T
    out.Bskel[3] = Usamp[3] @ h.B[3] @ Vsamp[2].T
    out.D = {tau: h.D[tau].copy() for tau in t.leaves()}
    return out


def _blkdiag(P, Q):
    M = np.zeros((P.shape[0] + Q.shape[0], P.shape[1] + Q.shape[1]))
    M[:P.shape[0], :P.shape[1]] = P
    M[P.shape[0]:, P.shape[1]:] = Q
    return M


def hbsid_apply(g: HBSID, X: np.ndarray, transpose: bool = False) -> np.ndarray:
    """Apply the HBS-ID form (partial-apply figure with interpolation matrices)."""
    t = g.tree
    Tin, Tout = (g.Tout, g.Tin) if transpose else (g.Tin, g.Tout)

    def Bs(a):
        return g.Bskel[a ^ 1].T if transpose else g.Bskel[a]

    qhat, uhat = {}, {}
    for tau in t.leaves():
        qhat[tau] = Tout[tau] @ X[t.rows(tau)]
    for lev in range(t.L - 1, 0, -1):
        for tau in t.level_nodes(lev):
            qhat[tau] = Tout[tau] @ np.vstack([qhat[2 * tau], qhat[2 * tau + 1]])
    uhat[2] = Bs(2) @ qhat[3]
    uhat[3] = Bs(3) @ qhat[2]
    for lev in range(1, t.L):
        for tau in t.level_nodes(lev):
            a, b = 2 * tau, 2 * tau + 1
            down = Tin[tau].T @ uhat[tau]
            ka = Tin[a].shape[0]
            uhat[a] = Bs(a) @ qhat[b] + down[:ka]
            uhat[b] = Bs(b) @ qhat[a] + down[ka:]
    Y = np.zeros_like(X, dtype=np.float64)
    for tau in t.leaves():
        I = t.rows(tau)
        Y[I] = Tin[tau].T @ uhat[tau] + (g.D[tau].T if transpose else g.D[tau]) @ X[I]
    return Y


def hbsid_dense(g: HBSID) -> np.ndarray:
    return hbsid_apply(g, np.eye(g.tree.N))
