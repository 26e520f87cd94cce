"""Oracle pins for HBS compression (Sec. 4.1-4.2), the partial apply A^(m)
(Fig. "Application of A^(m) in the HBS framework") and HBS-ID (Sec. 4.3)."""
import numpy as np
import pytest

import workloads as W
from oracle import hbs, hodlr
from oracle.tree import build_tree


def synthetic_hbs(N, m, k, seed):
    """Dense matrix with exact nested bases of rank k, built directly from the
    definition of Sec. 2.9 (long bases telescoped from random short ones)."""
    t = build_tree(N, m)
    rng = np.random.default_rng(seed)
    U, V = {}, {}
    for tau in t.leaves():
        U[tau] = rng.standard_normal((int(t.size[tau]), k))
        V[tau] = rng.standard_normal((int(t.size[tau]), k))
    for lev in range(t.L - 1, 0, -1):
        for tau in t.level_nodes(lev):
            a, b = 2 * tau, 2 * tau + 1
            for Lb in (U, V):
                S = rng.standard_normal((2 * k, k)) / np.sqrt(2 * k)
                Lb[tau] = np.vstack([Lb[a] @ S[:k], Lb[b] @ S[k:]])
    A = np.zeros((N, N))
    for lev in range(1, t.L + 1):
        for a in t.level_nodes(lev):
            A[t.rows(a), t.rows(a ^ 1)] = U[a] @ rng.standard_normal((k, k)) @ V[a ^ 1].T
    for tau in t.leaves():
        n = int(t.size[tau])
        A[t.rows(tau), t.rows(tau)] = rng.standard_normal((n, n))
    return A, t


@pytest.fixture(scope="module")
def exact():
    A, t = synthetic_hbs(512, 32, 5, seed=21)
    h = hbs.compress(hodlr.dense_apply_fn(A), t, r=15, seed=3)
    return A, t, h


@pytest.fixture(scope="module")
def logk():
    N = 1024
    A = W.log_kernel(N).astype(np.float64)
    t = build_tree(N, 64)
    h = hbs.compress(hodlr.dense_apply_fn(A), t, r=40, seed=2, mixed=True)
    return A, t, h


def test_exact_recovery(exact):
    A, t, h = exact
    assert np.linalg.norm(A - hbs.dense(h)) / np.linalg.norm(A) < 1e-12
    X = np.random.default_rng(1).standard_normal((t.N, 2))
    assert np.linalg.norm(hbs.apply(h, X, True) - A.T @ X) < 1e-11 * np.linalg.norm(A.T @ X)


def test_partial_apply_is_masked_matrix(exact):
    A, t, h = exact
    for m in range(t.L + 1):
        M = np.zeros_like(A)
        for j in range(1, m + 1):
            for a in t.level_nodes(j):
                M[t.rows(a), t.rows(a ^ 1)] = A[t.rows(a), t.rows(a ^ 1)]
        for tr in (False, True):
            P = hbs.partial_apply(h, m, np.eye(t.N), transpose=tr)
            assert np.linalg.norm(P - (M.T if tr else M)) <= 1e-11 * np.linalg.norm(A)


def test_nestedness_and_neutered_blocks(logk):
    A, t, h = logk
    r = h.r
    for lev in range(1, t.L):
        for tau in t.level_nodes(lev):
            a, b = 2 * tau, 2 * tau + 1
            U_tel = np.vstack([h.Ulong[a] @ h.Ushort[tau][:r], h.Ulong[b] @ h.Ushort[tau][r:]])
            # nested up to the sample weights y: directions below the noise level
            # of the samples need not telescope
            res = (h.Ulong[tau] - U_tel) * h.y[tau][None, :]
            assert np.linalg.norm(res) / np.linalg.norm(h.y[tau]) < 1e-7
    # the long basis spans the neutered row block A(I_tau, I_tau^c) (Sec. 2.9)
    for tau in list(t.level_nodes(2)) + list(t.leaves())[:4]:
        mask = np.ones(t.N, bool)
        mask[t.rows(tau)] = False
        blk = A[t.rows(tau)][:, mask]
        Ub = h.Ulong[tau]
        assert np.linalg.norm(blk - Ub @ (Ub.T @ blk)) / np.linalg.norm(blk) < 1e-7
        blkc = A[mask][:, t.rows(tau)]
        Vb = h.Vlong[tau]
        assert np.linalg.norm(blkc - (blkc @ Vb) @ Vb.T) / np.linalg.norm(blkc) < 1e-7


def test_hbs_accuracy_log_kernel(logk):
    A, t, h = logk
    assert np.linalg.norm(A - hbs.dense(h)) / np.linalg.norm(A) < 1e-7


def test_hbsid_skeleton_submatrix_and_interpolation(logk):
    A, t, h = logk
    g = hbs.to_hbsid(h, tol=1e-7)
    # Sec. 4.3: B_skel(a, b) equals the submatrix A(row skeleton of a, column skeleton of b)
    for a in [2, 3, 4, 5] + list(t.leaves())[:6]:
        sub = A[np.ix_(g.Iin[a], g.Iout[a ^ 1])]
        assert np.linalg.norm(g.Bskel[a] - sub) <= 1e-6 * np.linalg.norm(sub)
    # interpolation matrices contain the identity on the skeleton and stay bounded
    for tau in t.leaves():
        Tin = g.Tin[tau]
        J = g.Iin[tau] - int(t.start[tau])
        assert np.allclose(Tin[:, J], np.eye(Tin.shape[0]))
        assert np.max(np.abs(Tin)) <= 2.0
    # nested skeletons: the skeleton of a parent is taken from its children's
    for lev in range(1, t.L):
        for tau in t.level_nodes(lev):
            kids = set(g.Iin[2 * tau]) | set(g.Iin[2 * tau + 1])
            assert set(g.Iin[tau]) <= kids
    err = np.linalg.norm(A - hbs.hbsid_dense(g)) / np.linalg.norm(A)
    assert err < 1e-7
    assert max(g.rank_in(x) for x in g.Tin) <= h.r


def test_hbsid_transpose(logk):
    A, t, h = logk
    g = hbs.to_hbsid(h, tol=1e-7)
    X = np.random.default_rng(2).standard_normal((t.N, 2))
    assert np.linalg.norm(hbs.hbsid_apply(g, X, True) - hbs.hbsid_dense(g).T @ X) < 1e-12 * np.linalg.norm(A) * 10


def test_hbsid_exact_case_fixed_rank(exact):
    A, t, h = exact
    g = hbs.to_hbsid(h, tol=1e-12)
    assert max(g.rank_in(x) for x in g.Tin) == 5
    assert np.linalg.norm(A - hbs.hbsid_dense(g)) / np.linalg.norm(A) < 1e-10
