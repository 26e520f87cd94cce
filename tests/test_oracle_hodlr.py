"""Oracle pins for HODLR compression (Sec. 3, Fig. "Randomized compression of a
HODLR matrix") and the level-truncated apply A^(l) (Sec. 2.8)."""
import numpy as np
import pytest

import workloads as W
from oracle import hodlr
from oracle.lowrank import qr_basis
from oracle.tree import build_tree


@pytest.fixture(scope="module")
def exact_case():
    f = W.synthetic_hodlr_factors(512, 32, 6, seed=11, shift=512.0)
    A = W.dense_from_factors(f)
    t = build_tree(512, 32)
    h = hodlr.compress(hodlr.dense_apply_fn(A), t, r=16, k=6, seed=3)
    return A, t, h


def test_exact_recovery(exact_case):
    A, t, h = exact_case
    err = np.linalg.norm(A - hodlr.dense(h)) / np.linalg.norm(A)
    assert err < 1e-13


def test_config1_exact_recovery():
    f = W.synthetic_hodlr_factors(1024, 64, 10, seed=1, shift=1024.0)
    A = W.dense_from_factors(f)
    h = hodlr.compress(hodlr.dense_apply_fn(A), build_tree(1024, 64), r=20, k=10, seed=2)
    assert np.linalg.norm(A - hodlr.dense(h)) / np.linalg.norm(A) < 1e-13


def test_diagonal_blocks_exact(exact_case):
    A, t, h = exact_case
    for tau in t.leaves():
        I = t.rows(tau)
        assert np.linalg.norm(h.D[tau] - A[I, I]) <= 1e-12 * np.linalg.norm(A[I, I])


def test_transpose_apply(exact_case):
    A, t, h = exact_case
    X = np.random.default_rng(0).standard_normal((t.N, 3))
    assert np.allclose(hodlr.apply(h, X, transpose=True), A.T @ X, rtol=0, atol=1e-10 * np.abs(A).max())


def test_partial_apply_is_masked_matrix(exact_case):
    A, t, h = exact_case
    for level in range(t.L + 1):
        M = np.zeros_like(A)
        for j in range(1, level + 1):
            for a in t.level_nodes(j):
                M[t.rows(a), t.rows(a ^ 1)] = A[t.rows(a), t.rows(a ^ 1)]
        P = hodlr.partial_apply(h, level, np.eye(t.N))
        assert np.linalg.norm(P - M) <= 1e-12 * np.linalg.norm(A)


def test_tol_mode_ranks_equal_exact_rank():
    f = W.synthetic_hodlr_factors(512, 32, 5, seed=12, shift=0.0)
    A = W.dense_from_factors(f)
    h = hodlr.compress(hodlr.dense_apply_fn(A), build_tree(512, 32), r=15, tol=1e-10, seed=4)
    assert {h.rank(a) for a in h.U} == {5}


def test_log_kernel_ranks_match_dense_svd():
    N = 512
    A = W.log_kernel(N).astype(np.float64)
    t = build_tree(N, 32)
    h = hodlr.compress(hodlr.dense_apply_fn(A), t, r=40, tol=1e-7, seed=2)
    for j in range(1, t.L + 1):
        for a in t.level_nodes(j):
            s = np.linalg.svd(A[t.rows(a), t.rows(a ^ 1)], compute_uv=False)
            brute = int(np.count_nonzero(s > h.eps_abs))
            assert abs(h.rank(a) - brute) <= 2, (a, h.rank(a), brute)
    assert np.linalg.norm(A - hodlr.dense(h)) / np.linalg.norm(A) < 1e-7


def test_range_finder_bound():
    # Sec. 2.5: ||A - Q Q^* A|| <= (1 + 11 sqrt(k+p) sqrt(min(m, n))) sigma_{k+1}
    N, r, p = 1024, 20, 10
    A = W.log_kernel(N).astype(np.float64)
    t = build_tree(N, 64)
    X = hodlr.gaussian_test_matrix(t, 0, r, seed=5, mixed=False)
    Y = A @ X
    for node, cols, sib in ((2, slice(0, r), 3), (3, slice(r, 2 * r), 2)):
        blk = A[t.rows(node), t.rows(sib)]
        Q = qr_basis(Y[t.rows(node), cols])
        s = np.linalg.svd(blk, compute_uv=False)
        k = r - p
        bound = (1 + 11 * np.sqrt(k + p) * np.sqrt(min(blk.shape))) * s[k]
        assert np.linalg.norm(blk - Q @ (Q.T @ blk), 2) <= bound


@pytest.mark.parametrize("N,m", [(256, 16), (1024, 16), (4096, 16)])
def test_matvec_counts_linear_in_levels(N, m):
    f = W.synthetic_hodlr_factors(N, m, 3, seed=13, shift=float(N))
    t = build_tree(N, m)
    fn = lambda X, tr: W.dense_from_factors(f).T @ X if tr else None  # noqa: E731
    A = W.dense_from_factors(f)
    h = hodlr.compress(hodlr.dense_apply_fn(A), t, r=8, k=3, seed=1)
    assert h.cols_A == 2 * 8 * t.L + t.n_max
    assert h.cols_At == 2 * 8 * t.L


def test_mixed_test_matrix_is_bf16_exact():
    t = build_tree(300, 40)
    X = hodlr.gaussian_test_matrix(t, 2, 5, seed=1, mixed=True)
    bits = X.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    assert np.array_equal(X.astype(np.float32).astype(np.float64), X)
    # exactly r nonzeros per row (on the child's half)
    assert np.all(np.count_nonzero(X, axis=1) == 5)


def test_range_basis_reading_same_accuracy():
    """The numerical-range reading of qr(Y) reaches the same accuracy as the
    Householder reading and recovers exact-rank matrices to rounding."""
    f = W.synthetic_hodlr_factors(512, 32, 6, seed=11, shift=512.0)
    A = W.dense_from_factors(f)
    t = build_tree(512, 32)
    h = hodlr.compress(hodlr.dense_apply_fn(A), t, r=16, k=6, seed=3, basis="range")
    assert np.linalg.norm(A - hodlr.dense(h)) / np.linalg.norm(A) < 1e-13
    L = W.log_kernel(1024).astype(np.float64)
    t = build_tree(1024, 64)
    e = [np.linalg.norm(L - hodlr.dense(hodlr.compress(hodlr.dense_apply_fn(L), t, r=40, tol=1e-7,
                                                         seed=2, basis=b))) / np.linalg.norm(L)
         for b in ("qr", "range")]
    assert max(e) < 1e-7 and abs(e[0] - e[1]) < 0.5 * max(e)
