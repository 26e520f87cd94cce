"""Oracle pins for the factored HODLR apply and the gradients of ||Hx - b||^2."""
import numpy as np
import pytest

import workloads as W
from oracle import grad


@pytest.fixture(scope="module")
def case():
    f = W.synthetic_hodlr_factors(256, 32, 4, seed=5, shift=0.0)
    rng = np.random.default_rng(6)
    return f, rng.standard_normal(256), rng.standard_normal(256)


def test_apply_matches_dense(case):
    f, x, b = case
    H = W.dense_from_factors(f)
    assert np.allclose(grad.apply(f, x), H @ x, atol=1e-11)
    assert np.allclose(grad.apply(f, x, transpose=True), H.T @ x, atol=1e-11)


def test_dense_gradient(case):
    f, x, b = case
    H = W.dense_from_factors(f)
    dx, dU, dV, dD = grad.gradients(f, x, b)
    assert np.allclose(dx, 2 * H.T @ (H @ x - b), rtol=1e-12, atol=1e-9)


def _fd(fun, arr, idx, h):
    old = arr[idx]
    arr[idx] = old + h
    lp = fun()
    arr[idx] = old - h
    lm = fun()
    arr[idx] = old
    return (lp - lm) / (2 * h)


def test_central_differences(case):
    f, x, b = case
    f = {k: (v if not isinstance(v, list) else [None if a is None else a.copy() for a in v])
         for k, v in f.items()}
    x = x.copy()
    dx, dU, dV, dD = grad.gradients(f, x, b)
    rng = np.random.default_rng(0)
    fun = lambda: grad.loss(f, x, b)  # noqa: E731
    for i in rng.integers(0, 256, 5):
        fd = _fd(fun, x, int(i), 1e-5)
        assert abs(fd - dx[i]) <= 1e-6 * max(1.0, abs(dx[i]))
    for j in (1, f["L"]):
        for _ in range(3):
            idx = (int(rng.integers(0, 256)), int(rng.integers(0, 4)))
            assert abs(_fd(fun, f["U"][j], idx, 1e-5) - dU[j][idx]) <= 1e-6 * max(1.0, abs(dU[j][idx]))
            assert abs(_fd(fun, f["V"][j], idx, 1e-5) - dV[j][idx]) <= 1e-6 * max(1.0, abs(dV[j][idx]))
    for i in (0, 3):
        idx = (int(rng.integers(0, 32)), int(rng.integers(0, 32)))
        assert abs(_fd(fun, f["D"][i], idx, 1e-5) - dD[i][idx]) <= 1e-6 * max(1.0, abs(dD[i][idx]))
