"""Oracle pins for qr / svd / id (Secs. 2.2-2.4, 2.6)."""
import numpy as np
import pytest

from oracle.lowrank import fix_signs, interp_decomp, pivoted_qr, qr_basis, range_basis, svd_trunc


def _lowrank(m, n, k, seed, decay=1e-3):
    rng = np.random.default_rng(seed)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, min(m, n))))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, min(m, n))))
    s = np.array([1.0 if i < k else decay ** (1 + i - k) for i in range(min(m, n))])
    return (Q1 * s) @ Q2.T, s


def test_qr_basis_orthonormal_and_spanning():
    A, _ = _lowrank(50, 12, 12, 1)
    Q = qr_basis(A)
    assert np.allclose(Q.T @ Q, np.eye(12), atol=1e-14)
    assert np.linalg.norm(A - Q @ (Q.T @ A)) < 1e-13


def test_svd_eckart_young():
    A, s = _lowrank(40, 30, 5, 2, decay=1e-2)
    U, sv, Vt = svd_trunc(A, eps=1e-3)
    # eps mode: keep sigma > eps -> 5 + 1 terms (1e-2 > 1e-3 > 1e-4)
    assert sv.size == 6
    assert abs(np.linalg.norm(A - (U * sv) @ Vt, 2) - s[6]) < 1e-12
    U, sv, Vt = svd_trunc(A, k=3)
    assert sv.size == 3
    assert abs(np.linalg.norm(A - (U * sv) @ Vt, 2) - s[3]) < 1e-12


def test_pivoted_qr_matches_lapack_diagonal():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(3)
    A = rng.standard_normal((20, 35)) * np.logspace(0, -6, 35)[None, :]
    R, perm, rdiag = pivoted_qr(A)
    _, R2, perm2 = scipy_linalg.qr(A, pivoting=True, mode="economic")
    assert np.allclose(rdiag, np.abs(np.diag(R2)), rtol=1e-10)
    assert np.array_equal(perm[:20], perm2[:20])
    Q = qr_basis(A[:, perm])
    assert np.allclose(np.abs(Q.T @ A[:, perm]), np.abs(R), atol=1e-12)


def test_interp_decomp_properties():
    A, s = _lowrank(30, 60, 7, 4, decay=1e-4)
    J, T = interp_decomp(A, eps=1e-2)
    k = J.size
    assert k == 7
    assert np.allclose(T[:, J], np.eye(k), atol=1e-14)
    assert np.max(np.abs(T)) <= 2.0
    err = np.linalg.norm(A - A[:, J] @ T, 2)
    assert err <= np.sqrt(1 + k * (60 - k)) * 10 * s[7]
    J2, T2 = interp_decomp(A, k=3)
    assert J2.size == 3 and T2.shape == (3, 60)


def test_interp_decomp_brute_force_tiny():
    # rank-2 4x6 matrix: columns 0 and 3 span, ID must reproduce exactly
    a = np.array([1.0, 2.0, 0.0, -1.0])
    b = np.array([0.0, 1.0, 1.0, 3.0])
    A = np.stack([a, 2 * a, a + b, b, -b, 3 * a - 2 * b], axis=1)
    J, T = interp_decomp(A, eps=1e-12)
    assert J.size == 2
    assert np.allclose(A[:, J] @ T, A, atol=1e-13)


def test_range_basis_spans_numerical_range():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((80, 6)) @ rng.standard_normal((6, 20))  # rank 6 up to rounding
    Q = range_basis(A, rel_floor=1e-12)
    assert Q.shape[1] == 6
    assert np.allclose(Q.T @ Q, np.eye(6), atol=1e-14)
    assert np.linalg.norm(A - Q @ (Q.T @ A)) < 1e-12 * np.linalg.norm(A)
    Qf = qr_basis(A)
    assert np.linalg.norm(Qf @ (Qf.T @ Q) - Q) < 1e-12   # inside the span of the full Q
    Q0 = range_basis(A, rel_floor=1e-17)  # below rounding: noise directions are kept too
    assert 6 <= Q0.shape[1] <= 20 and np.allclose(Q0.T @ Q0, np.eye(Q0.shape[1]), atol=1e-13)
    assert range_basis(A).shape[1] == 6
    Z = np.zeros((10, 4))
    assert range_basis(Z).shape[1] == 0


def test_singular_vector_sign_convention_closed_form():
    """A = U0 diag(s0) V0^T with known factors whose right vectors already obey the
    convention: the oracle's svd must return U0 itself (not -U0 in any column),
    and every returned right vector must have a positive largest entry."""
    rng = np.random.default_rng(11)
    m, n = 30, 6
    U0, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V0, _ = np.linalg.qr(rng.standard_normal((n, n)))
    idx = np.argmax(np.abs(V0), axis=0)
    V0 = V0 * np.sign(V0[idx, np.arange(n)])[None, :]
    s0 = np.array([9.0, 5.0, 3.0, 2.0, 1.0, 0.5])
    A = U0 @ np.diag(s0) @ V0.T
    U, s, Vt = svd_trunc(A)
    assert np.allclose(s, s0, rtol=1e-13)
    assert np.allclose(U, U0, atol=1e-12)
    assert np.allclose(Vt, V0.T, atol=1e-12)
    Ur = range_basis(A)
    assert np.allclose(Ur, U0, atol=1e-12)
    # the convention itself, and that it keeps A = U S V^T
    B = rng.standard_normal((8, 5))
    Ub, sb, Vtb = np.linalg.svd(B, full_matrices=False)
    Uf, Vtf = fix_signs(-Ub, -Vtb)
    rows = np.arange(Vtf.shape[0])
    assert np.all(Vtf[rows, np.argmax(np.abs(Vtf), axis=1)] > 0)
    assert np.allclose(Uf @ np.diag(sb) @ Vtf, B, atol=1e-13)


def test_svd_r_floor_zeroes_rounding_level_directions():
    """hbs._svd_r(floor=True), the significant-range reading of svd(., r): a
    closed-form matrix with singular values 3, 1e-11 and 1e-14 (orthonormal
    factors built from Householder reflections) keeps the first two triplets
    (1e-11 > 1e-12 sigma_1) and returns the third as zero columns with a zero
    singular value; without the floor all three come back."""
    from oracle.hbs import _svd_r

    rng = np.random.default_rng(17)

    def reflector(n):
        v = rng.standard_normal(n)
        return np.eye(n) - 2.0 * np.outer(v, v) / (v @ v)

    Uf, Vf = reflector(9)[:, :3], reflector(5)[:, :3]
    s = np.array([3.0, 1e-11, 1e-14])
    M = (Uf * s) @ Vf.T
    U, sv, V = _svd_r(M, 3, floor=True)
    assert sv[0] == pytest.approx(3.0, rel=1e-14)
    assert sv[1] == pytest.approx(1e-11, rel=1e-3)
    assert sv[2] == 0.0
    assert np.all(U[:, 2] == 0.0) and np.all(V[:, 2] == 0.0)
    for j in range(2):  # kept triplets: the closed-form ones up to sign
        sg = np.sign(U[:, j] @ Uf[:, j])
        assert np.allclose(U[:, j], sg * Uf[:, j], atol=1e-4 if j else 1e-14)
        assert np.allclose(V[:, j], sg * Vf[:, j], atol=1e-4 if j else 1e-14)
    U2, sv2, V2 = _svd_r(M, 3, floor=False)
    assert sv2[2] > 0.0 and np.linalg.norm(U2[:, 2]) == pytest.approx(1.0)
