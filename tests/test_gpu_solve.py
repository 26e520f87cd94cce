"""Fast direct solver of a compressed HODLR matrix (recursive Sherman-Morrison-
Woodbury over the levels) through the C ABI, against the dense solve of the same
compressed matrix (np.linalg.solve of its reconstruction: the definition of
A_c^{-1} B), both products and transposes."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
DEV = "cuda:0"


def _setup(N, m, k, prec, shift):
    f = W.synthetic_hodlr_factors(N, m, k, seed=31, shift=shift)
    A = W.dense_from_factors(f)
    dtype = torch.float64 if prec != hm.HM_MIXED else torch.float32
    At = torch.from_numpy(A).to(DEV, torch.float64 if prec == hm.HM_FP64 else torch.float32)
    op = hm.hm_dense_operator_create(At, fp64_blocks=(prec == hm.HM_A32))
    h = hm.hm_compress_hodlr(op, hm.Tree(N, m), k=k, p=10, seed=2, prec=prec)
    Ac = torch.empty((N, N), device=DEV, dtype=dtype)
    hm.hm_reconstruct_block(h, 0, N, 0, N, Ac)
    torch.cuda.synchronize()
    return h, Ac.double().cpu().numpy().T, dtype


@pytest.mark.parametrize("N,m,k,prec,u", [(1024, 64, 10, 0, 1.1e-16), (3000, 100, 8, 0, 1.1e-16),
                                          (4096, 128, 12, 2, 1.1e-16), (2048, 64, 10, 1, 6e-8)])
def test_solve_matches_dense_solve(N, m, k, prec, u):
    h, Ac, dtype = _setup(N, m, k, prec, shift=float(N))
    hm.hm_hodlr_factorize(h)
    # a backward-stable solve is accurate to about cond(A_c) u; the bound allows 100x
    tol = 100.0 * np.linalg.cond(Ac) * u
    rng = np.random.default_rng(N + k)
    B = rng.standard_normal((N, 5))
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).to(DEV, dtype)
    for trans in (0, 1):
        X = torch.empty_like(Bd)
        hm.hm_solve(h, trans, Bd, X)
        torch.cuda.synchronize()
        want = np.linalg.solve(Ac.T if trans else Ac, Bd.double().cpu().numpy().T)
        got = X.double().cpu().numpy().T
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        res = np.linalg.norm((Ac.T if trans else Ac) @ got - Bd.double().cpu().numpy().T) / np.linalg.norm(B)
        print(f"N={N} prec={prec} trans={trans}: |x - x_dense| / |x_dense| {err:.2e}, residual "
              f"{res:.2e}, bound {tol:.1e}")
        assert err <= tol, (trans, err)


def test_solve_needs_factorization_and_refactorizes():
    h, Ac, dtype = _setup(512, 32, 5, hm.HM_FP64, shift=30.0)
    B = torch.ones((1, 512), device=DEV, dtype=torch.float64)
    X = torch.empty_like(B)
    with pytest.raises(hm.HmError) as e:
        hm.hm_solve(h, 0, B, X)
    assert e.value.status == 1
    hm.hm_hodlr_factorize(h)
    hm.hm_hodlr_factorize(h)  # again: the factors are rebuilt
    hm.hm_solve(h, 0, B, X)
    torch.cuda.synchronize()
    want = np.linalg.solve(Ac, np.ones(512))
    assert np.linalg.norm(X.cpu().numpy()[0] - want) <= 1e-12 * np.linalg.norm(want)


def _hodlr_from_dense(A, m, prec=0, **kw):
    At = torch.from_numpy(np.ascontiguousarray(A)).to(DEV, torch.float64)
    op = hm.hm_dense_operator_create(At)
    h = hm.hm_compress_hodlr(op, hm.Tree(A.shape[0], m), prec=prec, **kw)
    return h


def _dense(h, N):
    out = torch.empty((N, N), device=DEV, dtype=torch.float64)
    hm.hm_reconstruct_block(h, 0, N, 0, N, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().T


def test_product_of_compressed_operators_by_peeling():
    """Sec. 5.2's workflow on synthetic operators: compress I/2 + A1 (shifted
    black box over a handle), factorize it, then compress the product
    A2 (I/2 + A1)^{-1} by peeling through the apply of A2 and the solve, and the
    plain product A1 A2^T; each against the dense algebra of the handles."""
    N, m, k = 1024, 64, 4
    A1 = W.dense_from_factors(W.synthetic_hodlr_factors(N, m, k, seed=41, shift=float(N)))
    A2 = W.dense_from_factors(W.synthetic_hodlr_factors(N, m, k, seed=42, shift=1.0))
    h1 = _hodlr_from_dense(A1, m, k=k, p=10, seed=3)
    h2 = _hodlr_from_dense(A2, m, k=k, p=10, seed=4)
    A1c, A2c = _dense(h1, N), _dense(h2, N)
    t = hm.Tree(N, m)
    # I/2 + A1: a shifted black box over h1, compressed exactly (same ranks)
    sop = hm.hm_product_operator_create([h1], [hm.HM_FACTOR_APPLY], alpha=1.0, shift=0.5)
    hs = hm.hm_compress_hodlr(sop, t, k=k, p=10, seed=5, prec=0)
    Sc = _dense(hs, N)
    assert np.linalg.norm(Sc - (A1c + 0.5 * np.eye(N))) <= 1e-12 * np.linalg.norm(A1c)
    hm.hm_hodlr_factorize(hs)
    # A2 (I/2 + A1)^{-1}: numerically low rank off the diagonal, compressed to tol
    pop = hm.hm_product_operator_create([h2, hs], [hm.HM_FACTOR_APPLY, hm.HM_FACTOR_SOLVE])
    hp = hm.hm_compress_hodlr(pop, t, tol=1e-10, r=60, seed=6, prec=0)
    want = A2c @ np.linalg.inv(Sc)
    err = np.linalg.norm(_dense(hp, N) - want) / np.linalg.norm(want)
    print(f"A2 (I/2 + A1)^-1 compressed by peeling: rel err {err:.2e}, ranks "
          f"{hp.info['min_rank']}..{hp.info['max_rank']}")
    assert err <= 1e-9 and hp.info["saturated"] == 0
    # A1 A2^T: exact product, its transpose through the reversed factors
    qop = hm.hm_product_operator_create([h1, h2], [hm.HM_FACTOR_APPLY, hm.HM_FACTOR_TRANSPOSE])
    hq = hm.hm_compress_hodlr(qop, t, tol=1e-12, r=60, seed=7, prec=0)
    want = A1c @ A2c.T
    err = np.linalg.norm(_dense(hq, N) - want) / np.linalg.norm(want)
    print(f"A1 A2^T compressed by peeling: rel err {err:.2e}")
    assert err <= 1e-10
