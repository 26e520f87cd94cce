"""Parity at the full sizes of the measured workloads, through the C ABI.

The oracle cannot compress these sizes in seconds, so each test checks outputs
that the oracle side computes one by one, or properties that hold at any size:

* HBS-ID of the N = 65536 log kernel in the launch configuration the bench times
  (leaves 256, tol 1e-7, r = 60, HM_A32, tensor-core black box): the operator's
  entries against the kernel's formula, and sampled rows of A w, A^T w, and of
  the compressed H w, H^T w against FP64 row products of the formula's entries.
* HODLR of the N = 16384 log kernel (leaves 128, tol 1e-7, r = 60): the exact
  relative Frobenius error of the whole reconstructed matrix against the
  formula's N^2 entries, in HM_A32 and in HM_MIXED.
* The factored apply and adjoint at N = 262144, k = 32 (leaves 256): every
  output against the oracle's FP64 factored apply and gradients.
* The 64-operator batch (N log-uniform in [2048, 32768], k in [8, 40]): each
  handle's H w against the oracle's FP64 apply of the operator's own factors.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import grad as ograd

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
DEV = "cuda:0"


def _rows_rel(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def test_hbsid_a32_n65536_sampled_rows():
    N, m, tol, r = 65536, 256, 1e-7, 60
    A = torch.empty((N, N), device=DEV, dtype=torch.float32)
    hm.hm_gen_log_kernel(A)
    rng = np.random.default_rng(31)
    rows = np.sort(rng.choice(N, 48, replace=False))
    cols = np.sort(rng.choice(N, 1024, replace=False))
    # operator entries: the formula in FP64, rounded once to FP32 (a device log may
    # land on the other side of an FP32 rounding boundary: at most one ulp, rarely)
    want = W.log_kernel(N, rows, cols)
    got = A[torch.from_numpy(rows).to(DEV)][:, torch.from_numpy(cols).to(DEV)].cpu().numpy()
    ulp = np.abs(got.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1 and (ulp == 0).mean() > 0.99
    op = hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True)
    h = hm.hm_compress_hbs(op, hm.Tree(N, m), tol=tol, r=r, seed=2, prec=hm.HM_A32, hbs_id=1)
    assert h.info["saturated"] == 0
    w = rng.standard_normal((2, N))
    Arows = W.log_kernel(N, rows).astype(np.float64)          # 48 x N, the formula's rows
    want_rows = Arows @ w.T                                   # (A w)(rows); A is symmetric
    wd = torch.from_numpy(w).to(DEV)
    for trans in (0, 1):
        Yd, Yh = torch.empty_like(wd), torch.empty_like(wd)
        hm.hm_dense_apply(op, trans, wd, Yd)
        hm.hm_apply(h, trans, wd, Yh)
        torch.cuda.synchronize()
        yd = Yd.cpu().numpy()[:, rows].T
        yh = Yh.cpu().numpy()[:, rows].T
        # the black box: the split products of orders s + t >= 6 are not formed,
        # ~1e-8 relative per entry at worst
        assert _rows_rel(yd, want_rows) < 1e-7, trans
        # the compressed operator: the tolerance's scale (E measured ~2e-7 on unit vectors)
        assert _rows_rel(yh, want_rows) < 1e-6, trans
    # the metric's own property on the whole matrix (device reconstruction vs A)
    assert hm.hm_rel_frob_error(h, A) <= 1e-7


@pytest.mark.parametrize("N,seed", [(65536, 3), (65536, 4), (49152, 2)])
def test_hbsid_a32_tolerance_holds_at_other_seeds_and_sizes(N, seed):
    """The ID threshold scale (0.004 tol times the level-1 sample scale) was set on
    the measured N = 65536 workload with seed 2; the same configuration at other
    test-matrix seeds and at another N must stay within the tolerance over all N^2
    entries."""
    m, tol, r = 256, 1e-7, 60
    A = torch.empty((N, N), device=DEV, dtype=torch.float32)
    hm.hm_gen_log_kernel(A)
    op = hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True)
    h = hm.hm_compress_hbs(op, hm.Tree(N, m), tol=tol, r=r, seed=seed, prec=hm.HM_A32, hbs_id=1)
    err = hm.hm_rel_frob_error(h, A)
    print(f"HBS-ID N={N} seed={seed}: relative Frobenius error {err:.3e}, ranks "
          f"{h.info['min_rank']}..{h.info['max_rank']}, saturated {h.info['saturated']}")
    # at N = 49152 the leaves hold 192 points (arcs a third longer than the bench's):
    # the ID rank of a leaf near the ellipse's tips reaches 59-60 of r = 60 and may
    # saturate; the tolerance is then still checked over all N^2 entries
    if N == 65536:
        assert h.info["saturated"] == 0
    assert err <= tol


@pytest.mark.parametrize("prec,bound", [(2, 1e-7), (1, 1e-5)])
def test_hodlr_log_kernel_n16384_full_error(prec, bound):
    N, m, tol, r = 16384, 128, 1e-7, 60
    A = torch.empty((N, N), device=DEV, dtype=torch.float32)
    hm.hm_gen_log_kernel(A)
    if prec == hm.HM_A32:
        op = hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True)
    else:
        op = hm.hm_dense_operator_create(A)
    h = hm.hm_compress_hodlr(op, hm.Tree(N, m), tol=tol, r=r, seed=2, prec=prec)
    assert h.info["saturated"] == 0
    R = torch.empty((N, N), device=DEV, dtype=torch.float64 if prec != hm.HM_MIXED else torch.float32)
    hm.hm_reconstruct_block(h, 0, N, 0, N, R)     # column-major: R holds H^T row-major
    Hm = R.T.contiguous().double().cpu().numpy()
    del R
    Aw = W.log_kernel(N).astype(np.float64)          # the formula's N^2 entries
    err = float(np.linalg.norm(Hm - Aw) / np.linalg.norm(Aw))
    print(f"HODLR N={N} prec={prec}: relative Frobenius error {err:.3e}, ranks "
          f"{h.info['min_rank']}..{h.info['max_rank']}")
    assert err <= bound


def test_factored_apply_adjoint_n262144():
    N, m, k = 262144, 256, 32
    f = W.synthetic_hodlr_factors(N, m, k, seed=5, shift=0.0, dtype=np.float32)
    t = hm.Tree(N, m)
    L = f["L"]
    U = torch.from_numpy(np.stack([np.ascontiguousarray(f["U"][j].T) for j in range(1, L + 1)])).to(DEV)
    V = torch.from_numpy(np.stack([np.ascontiguousarray(f["V"][j].T) for j in range(1, L + 1)])).to(DEV)
    D = torch.from_numpy(np.stack([d.T.copy() for d in f["D"]])).to(DEV)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(N).astype(np.float32)
    b = rng.standard_normal(N).astype(np.float32)
    xd = torch.from_numpy(x).to(DEV)
    y, yt = torch.empty_like(xd), torch.empty_like(xd)
    hm.hm_hodlr_factored_apply(t, k, U, V, D, xd, y)
    hm.hm_hodlr_factored_apply(t, k, U, V, D, xd, yt, trans=1)
    res = y - torch.from_numpy(b).to(DEV)
    gx, gU, gV, gD = (torch.empty_like(a) for a in (xd, U, V, D))
    hm.hm_hodlr_factored_adjoint(t, k, U, V, D, xd, res, 2.0, gx, gU, gV, gD)
    torch.cuda.synchronize()
    x64, b64 = x.astype(np.float64), b.astype(np.float64)
    rel = lambda a, c: np.linalg.norm(a - c) / np.linalg.norm(c)  # noqa: E731
    assert rel(y.cpu().numpy(), ograd.apply(f, x64)) < 1e-5
    assert rel(yt.cpu().numpy(), ograd.apply(f, x64, transpose=True)) < 1e-5
    dx, dU, dV, dD = ograd.gradients(f, x64, b64)
    assert rel(gx.cpu().numpy(), dx) < 1e-5
    gUh, gVh, gDh = gU.cpu().numpy(), gV.cpu().numpy(), gD.cpu().numpy()
    for j in range(1, L + 1):
        assert rel(gUh[j - 1].T, dU[j]) < 1e-5, j
        assert rel(gVh[j - 1].T, dV[j]) < 1e-5, j
    num = sum(float(np.sum((gDh[i].T - d) ** 2)) for i, d in enumerate(dD))
    den = sum(float(np.sum(d ** 2)) for d in dD)
    assert (num / den) ** 0.5 < 1e-5
    # the fused training step the bench times, against the same oracle values
    y2 = torch.empty_like(xd)
    g2 = [torch.empty_like(a) for a in (xd, U, V, D)]
    hm.hm_hodlr_factored_loss_grad(t, k, U, V, D, xd, torch.from_numpy(b).to(DEV), 2.0, y2, None,
                                   *g2)
    torch.cuda.synchronize()
    assert rel(y2.cpu().numpy(), ograd.apply(f, x64)) < 1e-5
    assert rel(g2[0].cpu().numpy(), dx) < 1e-5
    gUh, gVh, gDh = g2[1].cpu().numpy(), g2[2].cpu().numpy(), g2[3].cpu().numpy()
    for j in range(1, L + 1):
        assert rel(gUh[j - 1].T, dU[j]) < 1e-5, j
        assert rel(gVh[j - 1].T, dV[j]) < 1e-5, j
    num = sum(float(np.sum((gDh[i].T - d) ** 2)) for i, d in enumerate(dD))
    assert (num / den) ** 0.5 < 1e-5


def test_batched_64_operators_against_factors():
    specs = W.batched_hodlr_specs(64)
    facs, mats, ops, trees, opts = [], [], [], [], []
    for sp in specs:
        N, k = sp["N"], sp["k"]
        f = W.synthetic_hodlr_factors(N, 64, k, seed=sp["op_seed"], shift=float(N), dtype=np.float32)
        A = torch.zeros((N, N), device=DEV, dtype=torch.float32)
        st, sz = f["start"], f["size"]
        for j in range(1, f["L"] + 1):
            Uj, Vj = torch.from_numpy(f["U"][j]).to(DEV), torch.from_numpy(f["V"][j]).to(DEV)
            for a in range(2 ** j, 2 ** (j + 1)):
                b = a ^ 1
                A[st[a]:st[a] + sz[a], st[b]:st[b] + sz[b]] = (
                    Uj[st[a]:st[a] + sz[a]].double() @ Vj[st[b]:st[b] + sz[b]].double().T).float()
        for i, t in enumerate(range(2 ** f["L"], 2 ** (f["L"] + 1))):
            A[st[t]:st[t] + sz[t], st[t]:st[t] + sz[t]] = torch.from_numpy(f["D"][i]).to(DEV)
        facs.append(f)
        mats.append(A)
        ops.append(hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True))
        trees.append(hm.Tree(N, 64))
        opts.append(dict(k=k, p=10, seed=sp["omega_seed"], prec=hm.HM_A32))
    hs = hm.hm_compress_batched(ops, trees, "hodlr", opts)
    rng = np.random.default_rng(41)
    worst = 0.0
    for i, (f, h) in enumerate(zip(facs, hs)):
        N = f["N"]
        assert h.info["max_rank"] == specs[i]["k"], i
        w = rng.standard_normal(N)
        Y = torch.empty((1, N), device=DEV, dtype=torch.float64)
        hm.hm_apply(h, 0, torch.from_numpy(w).to(DEV).reshape(1, N), Y)
        # the operator's own factors in FP64 (the device matrix rounds each entry
        # to FP32 once: ~6e-8 relative)
        e = _rows_rel(Y.cpu().numpy()[0], ograd.apply(f, w))
        worst = max(worst, e)
        assert e < 1e-5, (i, e)
    print(f"64 operators: worst relative error of H w {worst:.2e}")
