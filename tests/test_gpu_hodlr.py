"""GPU parity of the HODLR path (Sec. 3) against the FP64 oracle, through the
C ABI.  FP64 mode: 1e-12 relative Frobenius distance to the oracle's
reconstruction; mixed mode: 1e-6."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import grad as ograd
from oracle import hodlr as ohodlr
from oracle.philox import level_field
from oracle.tree import build_tree

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")

DEV = "cuda:0"


def colmajor(M: np.ndarray, dtype) -> torch.Tensor:
    """(ncols, n) device tensor holding the column-major n x ncols matrix M."""
    return torch.from_numpy(np.ascontiguousarray(M.T)).to(DEV, dtype)


def dense_from_handle(h, n, dtype):
    if h.info["prec"] == 2:
        dtype = torch.float64
    out = torch.empty((n, n), device=DEV, dtype=dtype)
    hm.hm_reconstruct_block(h, 0, n, 0, n, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy().T  # out holds column-major n x n


@pytest.mark.parametrize("prec", [0, 1])
def test_gaussian_test_matrix_matches_oracle(prec):
    N, m, r = 1000, 64, 11
    t = hm.Tree(N, m)
    ot = build_tree(N, m)
    for level in range(t.levels):
        X = torch.empty((2 * r, N), device=DEV, dtype=torch.float64 if prec == 0 else torch.float32)
        hm.hm_gaussian_test_matrix(t, level, r, 1234567, prec, X)
        torch.cuda.synchronize()
        got = X.double().cpu().numpy().T
        want = ohodlr.gaussian_test_matrix(ot, level, r, 1234567, mixed=(prec == 1))
        assert np.array_equal(got == 0, want == 0)
        if prec == 1:
            assert np.array_equal(got, want)  # BF16 values: bit-exact
        else:
            assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-300)) < 4e-15


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,ncols", [(1000, 37), (1024, 64), (300, 130)])
def test_dense_apply(dtype, N, ncols):
    rng = np.random.default_rng(N + ncols)
    A = rng.standard_normal((N, N))
    X = rng.standard_normal((N, ncols))
    X[: N // 3] = 0.0  # all-zero K-tiles are skipped
    At = torch.from_numpy(A).to(DEV, dtype)
    op = hm.hm_dense_operator_create(At)
    Xd = colmajor(X, dtype)
    for trans in (0, 1):
        Y = torch.empty((ncols, N), device=DEV, dtype=dtype)
        hm.hm_dense_apply(op, trans, Xd, Y)
        torch.cuda.synchronize()
        Aref = At.double().cpu().numpy()
        want = (Aref.T if trans else Aref) @ Xd.double().cpu().numpy().T
        got = Y.double().cpu().numpy().T
        tol = 1e-13 if dtype == torch.float64 else 2e-6
        assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


def _compress_dense(A, N, m, prec, **kw):
    dtype = torch.float64 if prec == 0 else torch.float32
    At = torch.from_numpy(np.ascontiguousarray(A)).to(DEV, dtype)
    op = hm.hm_dense_operator_create(At, fp64_blocks=(prec == 2))
    t = hm.Tree(N, m)
    h = hm.hm_compress_hodlr(op, t, prec=prec, **kw)
    return h, At, dtype


@pytest.mark.parametrize("N,m,k", [(1024, 64, 10), (1000, 64, 7), (700, 40, 5)])
def test_hodlr_fp64_exact_rank_parity(N, m, k):
    f = W.synthetic_hodlr_factors(N, m, k, seed=1, shift=float(N))
    A = W.dense_from_factors(f)
    h, At, dtype = _compress_dense(A, N, m, 0, k=k, p=10, seed=2)
    Ag = dense_from_handle(h, N, dtype)
    o = ohodlr.compress(ohodlr.dense_apply_fn(A), build_tree(N, m), r=k + 10, k=k, seed=2)
    Ao = ohodlr.dense(o)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(Ag - A) / nA < 1e-13          # exact recovery (Sec. 3)
    assert np.linalg.norm(Ag - Ao) / nA < 1e-12         # parity with the oracle
    info = h.info
    L = build_tree(N, m).L
    assert info["cols_A"] == 2 * (k + 10) * L + build_tree(N, m).n_max
    assert info["cols_At"] == 2 * (k + 10) * L
    assert info["max_rank"] == k and info["min_rank"] == k
    err = hm.hm_rel_frob_error(h, At)
    assert err < 1e-13


def test_hodlr_fp64_tol_mode_ranks():
    N, m, k = 512, 32, 5
    f = W.synthetic_hodlr_factors(N, m, k, seed=12, shift=0.0)
    A = W.dense_from_factors(f)
    h, At, dtype = _compress_dense(A, N, m, 0, tol=1e-10, r=15, seed=4)
    assert h.info["max_rank"] == k and h.info["min_rank"] == k
    assert hm.hm_rel_frob_error(h, At) < 1e-12


@pytest.mark.parametrize("N,m", [(2048, 128), (3000, 100)])
def test_hodlr_mixed_log_kernel_parity(N, m):
    A = W.log_kernel(N)
    h, At, dtype = _compress_dense(A, N, m, 1, tol=1e-7, r=60, seed=2)
    Ag = dense_from_handle(h, N, dtype)
    o = ohodlr.compress(ohodlr.dense_apply_fn(A), build_tree(N, m), r=60, tol=1e-7, seed=2, mixed=True)
    Ao = ohodlr.dense(o)
    A64 = A.astype(np.float64)
    nA = np.linalg.norm(A64)
    e_gpu = np.linalg.norm(Ag - A64) / nA
    e_par = np.linalg.norm(Ag - Ao) / nA
    print(f"N={N}: GPU err vs A {e_gpu:.3e}, vs oracle {e_par:.3e}, oracle err "
          f"{np.linalg.norm(Ao - A64) / nA:.3e}, ranks {h.info['min_rank']}..{h.info['max_rank']}")
    assert e_par < 1e-6
    assert e_gpu < 1e-6
    assert h.info["saturated"] == 0


def test_hodlr_apply_and_transpose_match_reconstruction():
    N, m = 1500, 64
    A = W.log_kernel(N).astype(np.float64)
    h, At, dtype = _compress_dense(A, N, m, 0, tol=1e-9, r=40, seed=3)
    Ag = dense_from_handle(h, N, dtype)
    X = np.random.default_rng(0).standard_normal((N, 5))
    for trans in (0, 1):
        Y = torch.empty((5, N), device=DEV, dtype=dtype)
        hm.hm_apply(h, trans, colmajor(X, dtype), Y)
        torch.cuda.synchronize()
        want = (Ag.T if trans else Ag) @ X
        assert np.linalg.norm(Y.cpu().numpy().T - want) <= 1e-12 * np.linalg.norm(want)
    # host-buffer entry point gives the same numbers
    Xh = torch.from_numpy(np.ascontiguousarray(X.T))
    Yh = torch.empty((5, N), dtype=torch.float64)
    hm.hm_apply_host(h, 0, Xh, Yh)
    assert np.linalg.norm(Yh.numpy().T - Ag @ X) <= 1e-12 * np.linalg.norm(Ag @ X)
    # ragged block reconstruction
    blk = torch.empty((77, 123), device=DEV, dtype=dtype)
    hm.hm_reconstruct_block(h, 100, 223, 900, 977, blk)
    torch.cuda.synchronize()
    assert np.allclose(blk.cpu().numpy().T, Ag[100:223, 900:977], rtol=0, atol=1e-13)


def test_callback_error_and_nonfinite():
    N, m = 256, 32
    t = hm.Tree(N, m)
    op = hm.callback_operator(N, lambda *a: 7)
    with pytest.raises(hm.HmError) as e:
        hm.hm_compress_hodlr(op, t, k=4, p=2, prec=0)
    assert e.value.status == 4
    A = np.eye(N)
    A[3, 200] = np.nan
    with pytest.raises(hm.HmError) as e:
        _compress_dense(A, N, m, 0, k=4, p=2)
    assert e.value.status == 6


@pytest.mark.parametrize("N,m,k", [(4096, 256, 8), (3000, 128, 5), (2048, 128, 48), (2050, 128, 33)])
def test_factored_apply_and_adjoint(N, m, k):
    """Oracle gradients; (2048, 48) and (2050, 33) take the k > 32 projection
    kernel, the latter with rows that are not 16-byte aligned (scalar loads)."""
    f = W.synthetic_hodlr_factors(N, m, k, seed=5, shift=0.0, dtype=np.float32)
    t = hm.Tree(N, m)
    L = f["L"]
    nmax = max(d.shape[0] for d in f["D"])
    U = torch.from_numpy(np.stack([np.ascontiguousarray(f["U"][j].T) for j in range(1, L + 1)])).to(DEV)
    V = torch.from_numpy(np.stack([np.ascontiguousarray(f["V"][j].T) for j in range(1, L + 1)])).to(DEV)
    Dp = np.zeros((len(f["D"]), nmax, nmax), np.float32)
    for i, d in enumerate(f["D"]):
        Dp[i, : d.shape[0], : d.shape[0]] = d.T  # column-major per leaf
    D = torch.from_numpy(Dp).to(DEV)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(N).astype(np.float32)
    b = rng.standard_normal(N).astype(np.float32)
    xd = torch.from_numpy(x).to(DEV)
    y = torch.empty_like(xd)
    hm.hm_hodlr_factored_apply(t, k, U, V, D, xd, y)
    yt = torch.empty_like(xd)
    hm.hm_hodlr_factored_apply(t, k, U, V, D, xd, yt, trans=1)
    torch.cuda.synchronize()
    want = ograd.apply(f, x.astype(np.float64))
    wantt = ograd.apply(f, x.astype(np.float64), transpose=True)
    assert np.linalg.norm(y.cpu().numpy() - want) <= 1e-5 * np.linalg.norm(want)
    assert np.linalg.norm(yt.cpu().numpy() - wantt) <= 1e-5 * np.linalg.norm(wantt)
    res = y - torch.from_numpy(b).to(DEV)
    gx, gU, gV, gD = (torch.full_like(a, float("nan")) for a in (xd, U, V, D))
    hm.hm_hodlr_factored_adjoint(t, k, U, V, D, xd, res, 2.0, gx, gU, gV, gD)
    torch.cuda.synchronize()
    dx, dU, dV, dD = ograd.gradients(f, x.astype(np.float64), b.astype(np.float64))
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)  # noqa: E731
    assert rel(gx.cpu().numpy(), dx) < 1e-5
    for j in range(1, L + 1):
        assert rel(gU[j - 1].cpu().numpy().T, dU[j]) < 1e-5
        assert rel(gV[j - 1].cpu().numpy().T, dV[j]) < 1e-5
    gDh = gD.cpu().numpy()
    for i, d in enumerate(dD):
        n = d.shape[0]
        assert rel(gDh[i, :n, :n].T, d) < 1e-5
        # the padding of a leaf smaller than n_max is written as zero (uneven leaves at N=3000)
        assert np.all(gDh[i, n:, :] == 0.0) and np.all(gDh[i, :, n:] == 0.0)
    # the fused training step (forward, residual, adjoint in one call, the forward's
    # projections reused) against the same oracle values
    bd = torch.from_numpy(b).to(DEV)
    y2, r2 = torch.full_like(xd, float("nan")), torch.full_like(xd, float("nan"))
    g2 = [torch.full_like(a, float("nan")) for a in (xd, U, V, D)]
    hm.hm_hodlr_factored_loss_grad(t, k, U, V, D, xd, bd, 2.0, y2, r2, *g2)
    torch.cuda.synchronize()
    assert np.linalg.norm(y2.cpu().numpy() - want) <= 1e-5 * np.linalg.norm(want)
    assert rel(r2.cpu().numpy(), want - b) < 1e-5
    assert rel(g2[0].cpu().numpy(), dx) < 1e-5
    for j in range(1, L + 1):
        assert rel(g2[1][j - 1].cpu().numpy().T, dU[j]) < 1e-5
        assert rel(g2[2][j - 1].cpu().numpy().T, dV[j]) < 1e-5
    gDh2 = g2[3].cpu().numpy()
    for i, d in enumerate(dD):
        n = d.shape[0]
        assert rel(gDh2[i, :n, :n].T, d) < 1e-5
        assert np.all(gDh2[i, n:, :] == 0.0) and np.all(gDh2[i, :, n:] == 0.0)
    # y and r may stay in scratch
    g3 = torch.full_like(xd, float("nan"))
    hm.hm_hodlr_factored_loss_grad(t, k, U, V, D, xd, bd, 2.0, None, None, g3)
    torch.cuda.synchronize()
    assert torch.equal(g3, g2[0])


def test_autograd_function_matches_adjoint():
    N, m, k = 1024, 64, 4
    f = W.synthetic_hodlr_factors(N, m, k, seed=8, shift=0.0, dtype=np.float32)
    t = hm.Tree(N, m)
    L = f["L"]
    U = torch.from_numpy(np.stack([np.ascontiguousarray(f["U"][j].T) for j in range(1, L + 1)])).to(DEV).requires_grad_()
    V = torch.from_numpy(np.stack([np.ascontiguousarray(f["V"][j].T) for j in range(1, L + 1)])).to(DEV).requires_grad_()
    D = torch.from_numpy(np.stack([d.T.copy() for d in f["D"]])).to(DEV).requires_grad_()
    x = torch.randn(N, device=DEV, generator=torch.Generator(DEV).manual_seed(1)).requires_grad_()
    b = torch.randn(N, device=DEV, generator=torch.Generator(DEV).manual_seed(2))
    y = hm.HodlrApply.apply(x, U, V, D, t, k)
    loss = ((y - b) ** 2).sum()
    loss.backward()
    dx, dU, dV, dD = ograd.gradients(f, x.detach().cpu().double().numpy(), b.cpu().double().numpy())
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)  # noqa: E731
    assert rel(x.grad.cpu().numpy(), dx) <= 1e-5
    for j in range(1, L + 1):
        assert rel(U.grad[j - 1].cpu().numpy().T, dU[j]) <= 1e-5
        assert rel(V.grad[j - 1].cpu().numpy().T, dV[j]) <= 1e-5
    gD = D.grad.cpu().numpy()
    for i, d in enumerate(dD):
        assert rel(gD[i].T, d) <= 1e-5


@pytest.mark.parametrize("N,m", [(2048, 128), (3000, 100)])
def test_hodlr_a32_log_kernel_parity(N, m):
    """FP32 operator applied in FP64 with an FP64 pipeline: the oracle's own arithmetic."""
    A = W.log_kernel(N)
    h, At, dtype = _compress_dense(A, N, m, 2, tol=1e-7, r=60, seed=2)
    Ag = dense_from_handle(h, N, torch.float64)
    # the GPU reads U = qr(Y) as an orthonormal basis of the numerical range of the
    # samples; the oracle run with the same reading is the parity reference
    o = ohodlr.compress(ohodlr.dense_apply_fn(A), build_tree(N, m), r=60, tol=1e-7, seed=2,
                        mixed=True, basis="range")
    Ao = ohodlr.dense(o)
    oq = ohodlr.compress(ohodlr.dense_apply_fn(A), build_tree(N, m), r=60, tol=1e-7, seed=2,
                         mixed=True)
    Aq = ohodlr.dense(oq)
    A64 = A.astype(np.float64)
    nA = np.linalg.norm(A64)
    e_gpu = np.linalg.norm(Ag - A64) / nA
    e_par = np.linalg.norm(Ag - Ao) / nA
    e_q = np.linalg.norm(Ag - Aq) / nA
    print(f"A32 N={N}: GPU err vs A {e_gpu:.3e}, vs oracle (range) {e_par:.3e}, vs oracle (qr) {e_q:.3e}")
    assert e_par < 1e-12
    assert e_q < 2 * max(e_gpu, np.linalg.norm(Aq - A64) / nA)  # within the truncation error
    assert e_gpu < 1e-7
    assert abs(hm.hm_rel_frob_error(h, At) - e_gpu) < 1e-9


def test_dense_apply_a32():
    N, c = 1000, 45
    rng = np.random.default_rng(3)
    A = rng.standard_normal((N, N)).astype(np.float32)
    X = rng.standard_normal((N, c))
    At = torch.from_numpy(A).to(DEV)
    op = hm.hm_dense_operator_create(At, fp64_blocks=True)
    Xd = colmajor(X, torch.float64)
    for trans in (0, 1):
        Y = torch.empty((c, N), device=DEV, dtype=torch.float64)
        hm.hm_dense_apply(op, trans, Xd, Y)
        torch.cuda.synchronize()
        A64 = A.astype(np.float64)
        want = (A64.T if trans else A64) @ X
        assert np.max(np.abs(Y.cpu().numpy().T - want)) <= 1e-13 * np.max(np.abs(want))


