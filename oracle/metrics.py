"""Error measures of Sec. 5.

* ``rel_frob``: ||A - A_c||_F / ||A||_F.
* ``estimate_E``: the randomized estimate E = max_i ||A w_i - A_c w_i|| / ||A w_i||
  over ten vectors w_i drawn uniformly from the unit sphere (normalized
  Gaussian vectors; the Gaussian entries come from the Philox stream reserved
  for the estimate, see ``oracle.philox``).

Pinned by tests/test_oracle_metrics.py: the vectors have unit length; E of an
exact representation is at rounding level; for A_c = (1 - d) A the estimate
is exactly d; E of a perturbation never exceeds ||A - A_c||_2 / sigma_min(A).
"""
from __future__ import annotations

import numpy as np

from .philox import STREAM_ESTIMATE, gaussian


def rel_frob(A: np.ndarray, Ac: np.ndarray) -> float:
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm(A - Ac) / np.linalg.norm(A))


def unit_vectors(N: int, count: int = 10, seed: int = 7) -> np.ndarray:
    W = gaussian(seed, STREAM_ESTIMATE, 0, np.arange(N), np.arange(count))
    return W / np.linalg.norm(W, axis=0, keepdims=True)


def estimate_E(apply_true, apply_comp, N: int, count: int = 10, seed: int = 7) -> float:
    W = unit_vectors(N, count, seed)
    Yt = apply_true(W)
    Yc = apply_comp(W)
    return float(np.max(np.linalg.norm(Yt - Yc, axis=0) / np.linalg.norm(Yt, axis=0)))
