"""qr / svd / id in the paper's three modes (Secs. 2.2, 2.3, 2.4 and 2.6).

Mode 1: full (economy) factorization.  Mode 2: an integer k, exactly k terms.
Mode 3: a real eps, the smallest number of terms whose truncation error is at
most eps.  As the paper does for small matrices, modes 2 and 3 call the full
LAPACK factorization and truncate it (Sec. 2.6).

Readings:
* ``svd(A, eps)`` keeps the singular values sigma_j > eps (eps is an absolute
  bound on the spectral truncation error, Eckart-Young, Sec. 2.3), at least one
  term; ``svd(A, k)`` keeps min(k, rank-dim) terms.
* The sign of each singular triplet (u_j, v_j) is free in the paper; it is
  fixed here: the largest-magnitude entry of v_j is positive (the first such
  entry on ties), see ``fix_signs``.  With packed test matrices the sample of
  one node carries the peel residual of other nodes in the same columns, so the
  result depends on these signs at the level of the truncation error; one
  convention makes it reproducible.
* ``id`` is computed from a column-pivoted Householder QR (Businger-Golub: at
  each step the remaining column of largest norm is moved to the front; on ties
  the lowest index wins), A(:, J) = Q R, rank k by |R_jj| > eps (mode 3) or k
  given (mode 2), then T = R11^{-1} [R11 R12] so that A ~= A(:, J(1:k)) T with
  T(:, J) = [I_k, R11^{-1} R12] in the original column order (Sec. 2.4: the
  ID "can be obtained from the full QR", Sec. 2.6).

Pinned by tests/test_oracle_lowrank.py (orthonormality, Eckart-Young error,
identity submatrix of the ID, |T| bound, ID error against sigma_{k+1}).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from . import cost


def qr_basis(A: np.ndarray) -> np.ndarray:
    """Q factor of the economy QR of A (orthonormal columns spanning range(A))."""
    Q, _ = cost.qr(A)
    return Q


def fix_signs(U: np.ndarray, Vt: np.ndarray):
    """Sign convention for singular triplets: flip (u_j, v_j) so that the
    largest-magnitude entry of the right singular vector v_j (row j of Vt) is
    positive; on ties the first such entry decides."""
    if Vt.shape[0] == 0:
        return U, Vt
    idx = np.argmax(np.abs(Vt), axis=1)  # argmax returns the first maximum
    sg = np.sign(Vt[np.arange(Vt.shape[0]), idx])
    sg[sg == 0] = 1.0
    return U * sg[None, :], Vt * sg[:, None]


RANGE_FLOOR = 1e-12


def range_basis(A: np.ndarray, rel_floor: float = RANGE_FLOOR) -> np.ndarray:
    """Orthonormal basis of the numerically significant range of A: the left
    singular vectors whose singular values exceed rel_floor * sigma_1.  A reading
    of "qr(Y)" for samples that are numerically rank deficient: it spans the
    significant part of the range of a full QR's Q and has no columns for
    directions at the rounding level, whose choice is arbitrary (they would pick
    up an arbitrary share of the coarser levels' truncation error through the
    transpose peel).  The default floor 1e-12 lies well above FP64 rounding and
    far below any compression tolerance."""
    U, s, Vt = cost.svd(A)
    U, Vt = fix_signs(U, Vt)
    if s.size == 0 or s[0] == 0.0:
        return U[:, :0]
    return U[:, : int(np.count_nonzero(s > rel_floor * s[0]))]


def svd_trunc(A: np.ndarray, k: int | None = None, eps: float | None = None):
    """[U, s, Vt] truncated per mode 2 (k) or mode 3 (eps); mode 1 if neither."""
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    U, Vt = fix_signs(U, Vt)
    n = s.size
    if k is not None:
        n = min(int(k), s.size)
    if eps is not None:
        keep = int(np.count_nonzero(s > eps))
        n = min(n, max(1, keep))
    return U[:, :n], s[:n], Vt[:n, :]


def pivoted_qr(A: np.ndarray, k_max: int | None = None):
    """Column-pivoted Householder QR (Businger-Golub): returns (R, perm, rdiag).

    R is min(m, n) x n upper trapezoidal for the permuted columns A[:, perm].
    Column norms are recomputed from the trailing block at every step (no
    downdating) so that the pivot choice is exactly "largest remaining norm,
    lowest index on ties".
    """
    R = np.array(A, dtype=np.float64, copy=True)
    m, n = R.shape
    perm = np.arange(n)
    steps = min(m, n) if k_max is None else min(m, n, int(k_max))
    rdiag = np.zeros(steps)
    for j in range(steps):
        norms = np.sum(R[j:, j:] ** 2, axis=0)
        p = j + int(np.argmax(norms))  # argmax returns the first maximum
        if p != j:
            R[:, [j, p]] = R[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        x = R[j:, j].copy()
        alpha = np.linalg.norm(x)
        if alpha == 0.0:
            rdiag[j] = 0.0
            continue
        if x[0] > 0:
            alpha = -alpha
        v = x
        v[0] -= alpha
        vnorm2 = float(v @ v)
        if vnorm2 > 0.0:
            R[j:, j:] -= np.outer(v, (2.0 / vnorm2) * (v @ R[j:, j:]))
        R[j, j] = alpha
        R[j + 1:, j] = 0.0
        rdiag[j] = abs(alpha)
    return R[:steps, :], perm, rdiag


def interp_decomp(A: np.ndarray, k: int | None = None, eps: float | None = None):
    """Column ID A ~= A[:, J] @ T (Sec. 2.4).  Returns (J, T) with T of shape k x n.

    Mode 2: k given.  Mode 3: k = number of |R_jj| > eps (at least 1).
    """
    m, n = A.shape
    R, perm, rdiag = pivoted_qr(A)
    steps = rdiag.size
    if k is None:
        k = int(np.count_nonzero(rdiag > (eps if eps is not None else 0.0)))
        k = max(1, k)
    k = min(int(k), steps, n)
    R11 = R[:k, :k]
    R12 = R[:k, k:]
    # T in pivoted order is [I, R11^{-1} R12]; scatter back to original order
    Tp = np.zeros((k, n))
    Tp[:, :k] = np.eye(k)
    if n > k:
        Tp[:, k:] = solve_triangular(R11, R12, lower=False)
    T = np.zeros((k, n))
    T[:, perm] = Tp
    return perm[:k].copy(), T
