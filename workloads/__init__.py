"""Seeded synthetic inputs shared by the oracle side and the device side.

This module holds none of the compression method's arithmetic: it only builds
the operators that the method is run on (its "black boxes") and the vectors of
the differentiation test.  Both the oracle tests and the device tests/bench take
their inputs from here, so both sides see the same bytes.

Operators
---------
* ``synthetic_hodlr_factors``: a seeded HODLR matrix with exact off-diagonal
  rank k.  For every sibling pair {a, b} the block A(I_a, I_b) = G_u G_v^T with
  G_u (n_a x k) and G_v (n_b x k) i.i.d. N(0, 1); every leaf block is
  N(0, 1) + shift * I.  Factors are returned level by level in "tall" arrays:
  U[level] and V[level] are N x k with rows I_a holding the factor of node a.
  Then A(I_a, I_b) = U[j][I_a] @ V[j][I_b]^T for siblings a, b on level j.
* ``dense_from_factors``: the dense N x N matrix of those factors.
* ``ellipse_points`` / ``log_kernel``: N points at uniform parameter
  t_i = 2 pi i / N on the ellipse (cos t, 0.5 sin t); entries
  log |x_i - x_j| computed in FP64 and rounded once to FP32, 1 on the diagonal.
"""
from __future__ import annotations

import numpy as np


def tree_ranges(N: int, leaf_size: int):
    """Uniform-depth tree (same rule as the method's tree): returns (L, start, size)."""
    L = 0
    while -(-N // 2 ** L) > leaf_size:
        L += 1
    start = np.zeros(2 ** (L + 1), np.int64)
    size = np.zeros(2 ** (L + 1), np.int64)
    size[1] = N
    for t in range(1, 2 ** L):
        n = int(size[t])
        start[2 * t], size[2 * t] = start[t], n // 2
        start[2 * t + 1], size[2 * t + 1] = start[t] + n // 2, n - n // 2
    return L, start, size


def synthetic_hodlr_factors(N: int, leaf_size: int, k: int, seed: int, shift: float,
                            dtype=np.float64):
    """Factors of a seeded exact-rank HODLR matrix (see module docstring).

    Returns dict(L, start, size, U=[L+1 arrays, index 0 unused], V=..., D=[leaf blocks]).
    """
    rng = np.random.default_rng(seed)
    L, start, size = tree_ranges(N, leaf_size)
    U = [None] + [rng.standard_normal((N, k)).astype(dtype) for _ in range(L)]
    V = [None] + [rng.standard_normal((N, k)).astype(dtype) for _ in range(L)]
    D = []
    for t in range(2 ** L, 2 ** (L + 1)):
        n = int(size[t])
        D.append((rng.standard_normal((n, n)) + shift * np.eye(n)).astype(dtype))
    return dict(L=L, start=start, size=size, U=U, V=V, D=D, k=k, N=N, leaf_size=leaf_size)


def dense_from_factors(f) -> np.ndarray:
    N, L, start, size = f["N"], f["L"], f["start"], f["size"]
    A = np.zeros((N, N))
    for j in range(1, L + 1):
        for a in range(2 ** j, 2 ** (j + 1)):
            b = a ^ 1
            ia = slice(start[a], start[a] + size[a])
            ib = slice(start[b], start[b] + size[b])
            A[ia, ib] = f["U"][j][ia].astype(np.float64) @ f["V"][j][ib].astype(np.float64).T
    for i, t in enumerate(range(2 ** L, 2 ** (L + 1))):
        it = slice(start[t], start[t] + size[t])
        A[it, it] = f["D"][i]
    return A


def ellipse_points(N: int) -> np.ndarray:
    t = 2.0 * np.pi * np.arange(N, dtype=np.float64) / N
    return np.stack([np.cos(t), 0.5 * np.sin(t)], axis=1)


def log_kernel(N: int, rows=None, cols=None) -> np.ndarray:
    """FP32 log-kernel entries A(rows, cols) (full matrix when rows/cols are None)."""
    x = ellipse_points(N)
    ri = np.arange(N) if rows is None else np.asarray(rows)
    ci = np.arange(N) if cols is None else np.asarray(cols)
    dx = x[ri, None, 0] - x[None, ci, 0]
    dy = x[ri, None, 1] - x[None, ci, 1]
    d = np.sqrt(dx * dx + dy * dy)
    with np.errstate(divide="ignore"):
        A = np.log(d)
    A[ri[:, None] == ci[None, :]] = 1.0
    return A.astype(np.float32)


def log_kernel_tables(N: int):
    """Tables of the matrix-free log kernel: S[m] = log|sin(pi m / N)| (m >= 1,
    S[0] unused) and P[s] = log(1 + 3 sin^2(pi s / N)) / 2 (s < 2N - 1), each FP64
    value kept as a float32 pair (hi, lo = remainder).  With d = pi (i - j) / N,
    f = pi (i + j) / N the ellipse points give
    |x_i - x_j|^2 = sin^2(d) (1 + 3 sin^2(f)).  Returns (Sh, Sl, Ph, Pl)."""
    m = np.arange(N, dtype=np.float64)
    with np.errstate(divide="ignore"):
        S = np.log(np.abs(np.sin(np.pi * m / N)))
    S[0] = 0.0
    t = np.arange(2 * N - 1, dtype=np.float64)
    sn = np.sin(np.pi * t / N)
    P = 0.5 * np.log1p(3.0 * sn * sn)
    Sh, Ph = S.astype(np.float32), P.astype(np.float32)
    Sl = (S - Sh.astype(np.float64)).astype(np.float32)
    Pl = (P - Ph.astype(np.float64)).astype(np.float32)
    return Sh, Sl, Ph, Pl


def log_kernel_tab(N: int, rows=None, cols=None, tables=None) -> np.ndarray:
    """Entries of the matrix-free log kernel: fl32(fl32(Sh + Ph) + fl32(Sl + Pl))
    off the diagonal (float32 arithmetic throughout), 1 on it."""
    Sh, Sl, Ph, Pl = tables if tables is not None else log_kernel_tables(N)
    ri = np.arange(N) if rows is None else np.asarray(rows)
    ci = np.arange(N) if cols is None else np.asarray(cols)
    d = np.abs(ri[:, None] - ci[None, :])
    s = ri[:, None] + ci[None, :]
    A = (Sh[d] + Ph[s]) + (Sl[d] + Pl[s])  # float32 + float32 -> float32
    A[d == 0] = np.float32(1.0)
    return A.astype(np.float32)


def batched_hodlr_specs(count: int = 64, seed: int = 4):
    """Sizes and ranks of the batched workload: N log-uniform in [2048, 32768]
    rounded to a multiple of 64, k uniform in [8, 40]; operator i is seeded 1000+i
    and its test matrices 2000+i."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        N = int(64 * round(np.exp(rng.uniform(np.log(2048), np.log(32768))) / 64))
        k = int(rng.integers(8, 41))
        specs.append(dict(N=N, k=k, op_seed=1000 + i, omega_seed=2000 + i))
    return specs
