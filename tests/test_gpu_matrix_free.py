"""The matrix-free log-kernel black box (entries formed inside the sampling
GEMM from two tables; Sec. 5: the black box is a fast multiplier, not a stored
matrix), through the C ABI:

* its entries equal the workload definition (FP32 sum of the two FP32 tables);
* its products equal the dense tensor-core engine's on the same entries, and
  the FP64 products of those entries to the engine's accuracy;
* an HBS-ID compression through it equals the compression through the dense
  operator holding the same entries;
* at N = 131072, twice the headline size, the compressions reach the noise
  floor that FP32 entries set for the method (about sqrt(L) x 3.4e-8), estimated
  on sampled rows against the entries.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
DEV = "cuda:0"


def _dense_entries(op, n):
    A = torch.empty((n, n), device=DEV, dtype=torch.float32)
    hm.hm_log_kernel_entries(op, 0, n, 0, n, A)
    torch.cuda.synchronize()
    return A


def test_entries_match_the_tables():
    N = 3000
    op = hm.hm_log_kernel_operator_create(N)
    rng = np.random.default_rng(4)
    rows = np.sort(rng.choice(N, 40, replace=False))
    A = _dense_entries(op, N).cpu().numpy()
    want = W.log_kernel_tab(N, rows)
    got = A[rows]
    # tables from the host's libm and numpy's: equal, or one FP32 ulp apart rarely
    ulp = np.abs(got.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1 and np.mean(ulp == 0) > 0.999, (ulp.max(), np.mean(ulp == 0))
    blk = torch.empty((5, 7), device=DEV, dtype=torch.float32)
    hm.hm_log_kernel_entries(op, 100, 105, 2990, 2997, blk)
    torch.cuda.synchronize()
    assert np.array_equal(blk.cpu().numpy(), A[100:105, 2990:2997])


@pytest.mark.parametrize("N,c", [(4096, 60), (3000, 37)])
def test_products_match_dense_engine(N, c):
    op = hm.hm_log_kernel_operator_create(N)
    A = _dense_entries(op, N)
    dense = hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True)
    rng = np.random.default_rng(N)
    X = rng.standard_normal((N, c))
    X[: N // 3] = 0.0  # all-zero K tiles are skipped by both
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(DEV)
    A64 = A.double().cpu().numpy()
    for trans in (0, 1):
        Ym, Yd = torch.empty_like(Xd), torch.empty_like(Xd)
        hm.hm_dense_apply(op, trans, Xd, Ym)
        hm.hm_dense_apply(dense, trans, Xd, Yd)
        hm.hm_dense_operator_check(op)
        got, ref = Ym.cpu().numpy().T, Yd.cpu().numpy().T
        want = (A64.T if trans else A64) @ X
        assert np.max(np.abs(got - ref)) <= 1e-15 * np.max(np.abs(want)), trans
        assert np.max(np.abs(got - want)) <= 3e-8 * np.max(np.abs(want)), trans


def test_compression_equals_dense_operator_compression():
    N, m, r = 8192, 256, 60
    op = hm.hm_log_kernel_operator_create(N)
    A = _dense_entries(op, N)
    dense = hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True)
    t = hm.Tree(N, m)
    kw = dict(tol=1e-7, r=r, seed=2, prec=hm.HM_A32, hbs_id=1)
    hmf = hm.hm_compress_hbs(op, t, **kw)
    hd = hm.hm_compress_hbs(dense, t, **kw)
    out = [torch.empty((N, N), device=DEV, dtype=torch.float64) for _ in range(2)]
    hm.hm_reconstruct_block(hmf, 0, N, 0, N, out[0])
    hm.hm_reconstruct_block(hd, 0, N, 0, N, out[1])
    torch.cuda.synchronize()
    diff = float((out[0] - out[1]).norm() / A.double().norm())
    err = hm.hm_rel_frob_error(hmf, A)
    print(f"N={N}: matrix-free vs dense-operator compression {diff:.3e}, error {err:.3e}")
    assert diff <= 1e-14
    assert err <= 1e-7
    assert hmf.info["cols_A"] == hd.info["cols_A"]


def _sampled_rows_error(op, h, N, seed=8, count=64):
    rows = np.sort(np.random.default_rng(seed).choice(N, count, replace=False))
    E = torch.zeros((count, N), device=DEV, dtype=torch.float64)
    E[torch.arange(count), torch.from_numpy(rows).to(DEV)] = 1.0
    Rc = torch.empty_like(E)
    hm.hm_apply(h, 1, E, Rc)  # rows of A_c = columns of A_c^T
    Ar = torch.empty((count, N), device=DEV, dtype=torch.float32)
    for q, i in enumerate(rows):
        hm.hm_log_kernel_entries(op, int(i), int(i) + 1, 0, N, Ar[q:q + 1])
    torch.cuda.synchronize()
    return float((Rc - Ar.double()).norm() / Ar.double().norm())


def test_n131072_reaches_the_fp32_noise_floor():
    """Twice the headline size.  The operator's entries are FP32 numbers: their
    rounding (relative 2^-24 / sqrt(3) RMS, about 3.4e-8) is full-rank noise in
    every off-diagonal block, and each of the L levels of peeling leaves its
    share of it in the finer levels' samples, so the relative Frobenius error of
    a compression settles near sqrt(L) x 3.4e-8 however tight the tolerance
    (measured: 9.1e-8 at N = 65536, L = 8, for both this operator and the dense
    one; about 1.1e-7 at N = 131072, L = 9, for tol from 1e-8 down to 3e-9).
    The HODLR form at tol 1e-8, r = 100 reaches that floor; the bound allows
    1.5 x the floor."""
    N, m = 131072, 256
    op = hm.hm_log_kernel_operator_create(N)
    t = hm.Tree(N, m)
    floor = np.sqrt(t.levels) * 2.0 ** -24 / np.sqrt(3.0)
    h = hm.hm_compress_hodlr(op, t, tol=1e-8, r=100, seed=2, prec=hm.HM_A32)
    est = _sampled_rows_error(op, h, N)
    print(f"N={N} HODLR: sampled-row relative Frobenius error {est:.3e} (floor {floor:.2e}), ranks "
          f"{h.info['min_rank']}..{h.info['max_rank']}, {h.info['t_compress_ms']:.1f} ms")
    assert h.info["saturated"] == 0
    assert est <= 1.5 * floor
    del h
    hb = hm.hm_compress_hbs(op, t, tol=1e-7, r=64, seed=2, prec=hm.HM_A32, hbs_id=1)
    eb = _sampled_rows_error(op, hb, N)
    print(f"N={N} HBS-ID r=64: sampled-row relative Frobenius error {eb:.3e}, saturated "
          f"{hb.info['saturated']}")
    assert eb <= 2.0 * floor
