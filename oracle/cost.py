"""Operation counts of the oracle's own arithmetic (T_net of Sec. 5, counted in
floating-point operations instead of timed).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  The paper states the cost
of a compression outside the black box as O(k^2 N log^2 N) for HODLR (Sec. 3.1:
the peel at level l applies l levels of factors) and O(k^2 N log N) for HBS
(Sec. 4.4: the nested partial apply touches one level of long bases plus short
bases).  The oracle routes its dense products and factorizations through the
three helpers below, which compute exactly what NumPy would and add the textbook
operation count of each call to ``COUNT`` (products: 2 m n k; QR of an m x n
panel: 2 m n^2 - 2 n^3 / 3; SVD of an m x n panel, m >= n: the R-SVD count
4 m n^2 + 22 n^3 of Golub and Van Loan, Matrix Computations, 4th ed., Fig. 8.6.1
for U, S and V).  ``tests/test_oracle_cost.py`` pins the scaling laws on these
counts.
"""
from __future__ import annotations

import numpy as np


class _Count:
    flops: float = 0.0


COUNT = _Count()


def reset() -> None:
    COUNT.flops = 0.0


def mm(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A @ B, counted as 2 m n k."""
    n = B.shape[1] if B.ndim == 2 else 1
    COUNT.flops += 2.0 * A.shape[0] * A.shape[1] * n
    return A @ B


def svd(M: np.ndarray):
    """Economy SVD (np.linalg.svd, full_matrices=False), counted by the R-SVD formula."""
    m, n = M.shape
    a, b = max(m, n), min(m, n)
    COUNT.flops += 4.0 * a * b * b + 22.0 * b ** 3
    return np.linalg.svd(M, full_matrices=False)


def qr(M: np.ndarray):
    """Economy QR (np.linalg.qr, mode "reduced"), counted as Householder QR plus forming Q."""
    m, n = M.shape
    b = min(m, n)
    COUNT.flops += 2.0 * (2.0 * m * b * b - 2.0 * b ** 3 / 3.0)
    return np.linalg.qr(M, mode="reduced")
