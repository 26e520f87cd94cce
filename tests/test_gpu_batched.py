"""hm_compress_batched: many independent operators of uneven size and rank in one
call, through the C ABI, against one hm_compress_* call per operator (the same
hot path) and against the operators themselves."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
DEV = "cuda:0"


def dense_of(h, N, dtype=torch.float64):
    out = torch.empty((N, N), device=DEV, dtype=dtype)
    hm.hm_reconstruct_block(h, 0, N, 0, N, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().T


SPECS = [(640, 4), (1024, 10), (896, 6), (2048, 12), (1536, 8), (960, 5)]


def _check_batched(fmt, mats, ops, trees, opts, err_bound, ranks=None):
    hs = hm.hm_compress_batched(ops, trees, fmt, opts, max_concurrency=4)
    assert len(hs) == len(mats)
    for i, A in enumerate(mats):
        N = A.shape[0]
        one = (hm.hm_compress_hodlr if fmt == "hodlr" else hm.hm_compress_hbs)(ops[i], trees[i], **opts[i])
        Ab, A1 = dense_of(hs[i], N), dense_of(one, N)
        nA = np.linalg.norm(A)
        assert np.linalg.norm(Ab - A1) / nA < 1e-14, i
        assert np.linalg.norm(Ab - A) / nA < err_bound, i
        if ranks is not None:
            assert hs[i].info["max_rank"] == ranks[i]


def test_batched_hodlr_matches_one_call_per_operator():
    """Exact-rank synthetic HODLR operators of uneven size and rank (leaves of 64)."""
    m = 64
    mats, ops, trees, opts = [], [], [], []
    for i, (N, k) in enumerate(SPECS):
        A = W.dense_from_factors(W.synthetic_hodlr_factors(N, m, k, seed=1000 + i, shift=float(N)))
        mats.append(A)
        ops.append(hm.hm_dense_operator_create(torch.from_numpy(A).to(DEV)))
        trees.append(hm.Tree(N, m))
        opts.append(dict(k=k, p=10, seed=2000 + i, prec=hm.HM_FP64))
    _check_batched("hodlr", mats, ops, trees, opts, 1e-10, ranks=[k for _, k in SPECS])


def test_batched_mixed_panel_widths_eight_threads():
    """Sixteen operators whose panel widths k + p all differ, eight at a time: the
    QR and Jacobi kernels size their shared memory by the panel width, so this is
    where threads that configure one kernel for different widths would collide.
    Every handle must equal the one-call result."""
    m = 64
    rng = np.random.default_rng(7)
    mats, ops, trees, opts = [], [], [], []
    for i in range(16):
        N = int(64 * rng.integers(48, 97))
        k = 6 + 2 * i
        A = torch.from_numpy(W.dense_from_factors(
            W.synthetic_hodlr_factors(N, m, k, seed=3000 + i, shift=float(N)))).to(DEV)
        mats.append(A)
        ops.append(hm.hm_dense_operator_create(A))
        trees.append(hm.Tree(N, m))
        opts.append(dict(k=k, p=10, seed=4000 + i, prec=hm.HM_FP64))
    hs = hm.hm_compress_batched(ops, trees, "hodlr", opts, max_concurrency=8)
    for i, A in enumerate(mats):
        N = A.shape[0]
        one = hm.hm_compress_hodlr(ops[i], trees[i], **opts[i])
        Rb = torch.empty((N, N), device=DEV, dtype=torch.float64)
        R1 = torch.empty_like(Rb)
        hm.hm_reconstruct_block(hs[i], 0, N, 0, N, Rb)
        hm.hm_reconstruct_block(one, 0, N, 0, N, R1)
        nA = float(A.norm())
        assert float((Rb - R1).norm()) / nA < 1e-14, i
        assert float((Rb.T - A).norm()) / nA < 1e-10, i


def test_batched_hbsid_matches_one_call_per_operator():
    """Log-kernel operators of uneven size, tolerance mode (HBS nested bases)."""
    m = 128
    mats, ops, trees, opts = [], [], [], []
    for i, N in enumerate((1024, 1536, 2048, 1280)):
        A = W.log_kernel(N).astype(np.float64)
        mats.append(A)
        ops.append(hm.hm_dense_operator_create(torch.from_numpy(A).to(DEV)))
        trees.append(hm.Tree(N, m))
        opts.append(dict(tol=1e-7, r=40, seed=2000 + i, prec=hm.HM_FP64))
    _check_batched("hbsid", mats, ops, trees, opts, 1e-7)


def test_batched_error_names_the_operator():
    N, m = 512, 64
    A = torch.eye(N, device=DEV, dtype=torch.float64)
    good = hm.hm_dense_operator_create(A)
    bad = hm.callback_operator(N, lambda *a: 7)
    with pytest.raises(hm.HmError, match="operator 1") as e:
        hm.hm_compress_batched([good, bad, good], [hm.Tree(N, m)] * 3, "hodlr",
                               [dict(k=4, p=2, prec=hm.HM_FP64)] * 3)
    assert e.value.status == 4


def test_batched_empty():
    assert hm.hm_compress_batched([], [], "hodlr") == []


def test_batched_a32_level_wide_launches_equal_one_call():
    """HM_A32, the batch workload's precision: the TSQR rounds and the panel SVD of
    a level run as one launch over every operator's nodes (operators of uneven N,
    depth and panel width).  Each node's arithmetic is that of the one-operator
    call, so every handle must equal the one-call result bit for bit, with fewer
    launches than the one-operator calls together."""
    m = 64
    rng = np.random.default_rng(11)
    ops, trees, opts, keep = [], [], [], []
    for i in range(10):
        N = int(64 * rng.integers(16, 97))
        k = 4 + 3 * i
        A = torch.from_numpy(W.dense_from_factors(W.synthetic_hodlr_factors(
            N, m, k, seed=5000 + i, shift=float(N))).astype(np.float32)).to(DEV)
        keep.append(A)
        ops.append(hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True))
        trees.append(hm.Tree(N, m))
        opts.append(dict(k=k, p=10, seed=6000 + i, prec=hm.HM_A32))
    ones = [hm.hm_compress_hodlr(ops[i], trees[i], **opts[i]) for i in range(len(ops))]
    torch.cuda.synchronize()
    n0 = hm.hm_launch_count()
    ones = [hm.hm_compress_hodlr(ops[i], trees[i], **opts[i]) for i in range(len(ops))]
    torch.cuda.synchronize()
    n_one = hm.hm_launch_count() - n0
    n0 = hm.hm_launch_count()
    hs = hm.hm_compress_batched(ops, trees, "hodlr", opts, max_concurrency=4)
    torch.cuda.synchronize()
    n_batch = hm.hm_launch_count() - n0
    assert n_batch < n_one, (n_batch, n_one)
    for i, A in enumerate(keep):
        N = A.shape[0]
        Rb = torch.empty((N, N), device=DEV, dtype=torch.float64)
        R1 = torch.empty_like(Rb)
        hm.hm_reconstruct_block(hs[i], 0, N, 0, N, Rb)
        hm.hm_reconstruct_block(ones[i], 0, N, 0, N, R1)
        torch.cuda.synchronize()
        assert torch.equal(Rb, R1), i
        assert hs[i].info["max_rank"] == ones[i].info["max_rank"], i
        nA = float(A.double().norm())
        assert float((Rb.T - A.double()).norm()) / nA < 1e-6, i


def test_tune_batched_concurrency():
    """hm_tune_batched times the batch once per candidate concurrency and picks
    the fastest; the handles do not depend on the concurrency, so a batch run
    at the chosen value and at another one give the same matrices bit for bit."""
    m = 64
    ops, trees, opts, keep = [], [], [], []
    for i, (N, k) in enumerate(SPECS):
        A = torch.from_numpy(W.dense_from_factors(W.synthetic_hodlr_factors(
            N, m, k, seed=1000 + i, shift=float(N))).astype(np.float32)).to(DEV)
        keep.append(A)
        ops.append(hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True))
        trees.append(hm.Tree(N, m))
        opts.append(dict(k=k, p=10, seed=2000 + i, prec=hm.HM_A32))
    best, ms = hm.hm_tune_batched(ops, trees, "hodlr", opts, candidates=(1, 2, 4))
    assert best in (1, 2, 4) and set(ms) == {1, 2, 4}
    assert all(v > 0.0 for v in ms.values()) and ms[best] == min(ms.values())
    other = 1 if best != 1 else 4
    hb = hm.hm_compress_batched(ops, trees, "hodlr", opts, max_concurrency=best)
    ho = hm.hm_compress_batched(ops, trees, "hodlr", opts, max_concurrency=other)
    for i, (N, _) in enumerate(SPECS):
        assert np.array_equal(dense_of(hb[i], N), dense_of(ho[i], N)), i
    with pytest.raises(hm.HmError):
        hm.hm_tune_batched(ops, trees, "hodlr", opts, candidates=(0,))
