"""Oracle pins for the error measures of Sec. 5."""
import numpy as np

from oracle import metrics


def test_unit_vectors():
    W = metrics.unit_vectors(500)
    assert W.shape == (500, 10)
    assert np.allclose(np.linalg.norm(W, axis=0), 1.0)


def test_estimate_exact_and_scaled():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((300, 300))
    E0 = metrics.estimate_E(lambda W: A @ W, lambda W: A @ W, 300)
    assert E0 == 0.0
    d = 1e-5
    Ed = metrics.estimate_E(lambda W: A @ W, lambda W: (1 - d) * (A @ W), 300)
    assert abs(Ed - d) < 1e-15
    P = 1e-6 * rng.standard_normal((300, 300))
    Ep = metrics.estimate_E(lambda W: A @ W, lambda W: (A + P) @ W, 300)
    s = np.linalg.svd(A, compute_uv=False)
    assert Ep <= np.linalg.norm(P, 2) / s[-1]


def test_rel_frob():
    A = np.eye(4)
    assert metrics.rel_frob(A, 0.5 * A) == 0.5
