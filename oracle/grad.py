"""Factored HODLR apply, its transpose, and the gradients of the loss
L(x, U, V, D) = ||H x - b||^2 (differentiation line of the build; the apply is
the HODLR matrix-vector product of Sec. 2.8, O(k N log N)).

H is held as in ``workloads.synthetic_hodlr_factors``: for every level j = 1..L
the tall arrays U[j], V[j] (N x k; rows I_a hold the factor of node a) with
H(I_a, I_b) = U[j][I_a] V[j][I_b]^T for the siblings a, b of level j (sibling
matrix B = I_k), and a dense block D_tau for every leaf.

With res = H x - b:
  dL/dx          = 2 H^T res
  dL/dU[j][I_a]  = 2 res(I_a) (V[j][I_b]^T x(I_b))^T
  dL/dV[j][I_b]  = 2 x(I_b) (U[j][I_a]^T res(I_a))^T
  dL/dD_tau      = 2 res(I_tau) x(I_tau)^T

Pinned by tests/test_oracle_grad.py: central finite differences in FP64 for
every argument, and the dense gradient 2 H^T (H x - b) of the assembled matrix.
"""
from __future__ import annotations

import numpy as np


def _pairs(f):
    L, start, size = f["L"], f["start"], f["size"]
    for j in range(1, L + 1):
        for a in range(2 ** j, 2 ** (j + 1)):
            b = a ^ 1
            yield j, slice(start[a], start[a] + size[a]), slice(start[b], start[b] + size[b])


def _leaves(f):
    L, start, size = f["L"], f["start"], f["size"]
    for i, t in enumerate(range(2 ** L, 2 ** (L + 1))):
        yield i, slice(start[t], start[t] + size[t])


def apply(f, x: np.ndarray, transpose: bool = False) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    for j, ia, ib in _pairs(f):
        U = f["U"][j].astype(np.float64)
        V = f["V"][j].astype(np.float64)
        if not transpose:
            y[ia] += U[ia] @ (V[ib].T @ x[ib])
        else:
            y[ib] += V[ib] @ (U[ia].T @ x[ia])
    for i, it in _leaves(f):
        D = f["D"][i].astype(np.float64)
        y[it] += (D.T if transpose else D) @ x[it]
    return y


def loss(f, x, b) -> float:
    res = apply(f, x) - b
    return float(res @ res)


def gradients(f, x, b):
    """Returns (dx, dU, dV, dD) with dU/dV lists indexed like f["U"]."""
    x = np.asarray(x, dtype=np.float64)
    res = apply(f, x) - np.asarray(b, dtype=np.float64)
    dx = 2.0 * apply(f, res, transpose=True)
    dU = [None] + [np.zeros((f["N"], f["k"])) for _ in range(f["L"])]
    dV = [None] + [np.zeros((f["N"], f["k"])) for _ in range(f["L"])]
    for j, ia, ib in _pairs(f):
        U = f["U"][j].astype(np.float64)
        V = f["V"][j].astype(np.float64)
        dU[j][ia] += 2.0 * np.outer(res[ia], V[ib].T @ x[ib])
        dV[j][ib] += 2.0 * np.outer(x[ib], U[ia].T @ res[ia])
    dD = [2.0 * np.outer(res[it], x[it]) for _, it in _leaves(f)]
    return dx, dU, dV, dD
