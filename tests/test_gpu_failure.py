"""Failure statuses the C ABI declares, produced on the GPU without faulting it.

* HM_ETIMEOUT: the tensor-core GEMMs' pipeline waits are bounded by a
  host-settable poll limit (hm_set_wait_limit).  With a limit of one poll the
  first wait runs out; the block then lets its own copies and MMAs complete
  (those waits keep the full limit), writes NaN and raises the operator's
  flag, which the compress call and hm_dense_operator_check report.  The next
  call with the default limit on the same stream is exact again.
* HM_ERANK_SATURATED: in strict mode an adaptive rank that reaches r is an
  error (Sec. 2.5: the range finder is certified only for ranks below r).
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
DEV = "cuda:0"


@pytest.fixture
def default_limit():
    yield
    hm.hm_set_wait_limit(0)


def test_timeout_in_dense_apply_then_recovery(default_limit):
    N, c = 1024, 40
    rng = np.random.default_rng(11)
    A = rng.standard_normal((N, N)).astype(np.float32)
    X = rng.standard_normal((N, c))
    At = torch.from_numpy(A).to(DEV)
    op = hm.hm_dense_operator_create(At, fp64_blocks=True, tensor_cores=True)
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(DEV)
    Y = torch.empty((c, N), device=DEV, dtype=torch.float64)
    hm.hm_dense_apply(op, 0, Xd, Y)          # first use records the operator's scales
    hm.hm_dense_operator_check(op)
    hm.hm_set_wait_limit(1)
    hm.hm_dense_apply(op, 0, Xd, Y)
    with pytest.raises(hm.HmError) as e:
        hm.hm_dense_operator_check(op)
    assert e.value.status == 7  # HM_ETIMEOUT
    assert torch.isnan(Y).any()
    hm.hm_set_wait_limit(0)
    for trans in (0, 1):
        hm.hm_dense_apply(op, trans, Xd, Y)
        hm.hm_dense_operator_check(op)
        want = (A.astype(np.float64).T if trans else A.astype(np.float64)) @ X
        assert np.max(np.abs(Y.cpu().numpy().T - want)) <= 3e-8 * np.max(np.abs(want))


def test_timeout_in_compression_then_recovery(default_limit):
    N, m = 2048, 128
    A = W.log_kernel(N)
    At = torch.from_numpy(A).to(DEV)
    op = hm.hm_dense_operator_create(At, fp64_blocks=True, tensor_cores=True)
    t = hm.Tree(N, m)
    hm.hm_set_wait_limit(1)
    with pytest.raises(hm.HmError) as e:
        hm.hm_compress_hodlr(op, t, tol=1e-7, r=40, seed=2, prec=hm.HM_A32)
    assert e.value.status == 7
    hm.hm_set_wait_limit(0)
    h = hm.hm_compress_hodlr(op, t, tol=1e-7, r=40, seed=2, prec=hm.HM_A32)
    assert hm.hm_rel_frob_error(h, At) < 1e-7


def test_strict_rank_hodlr():
    N, m, k = 1024, 64, 16
    f = W.synthetic_hodlr_factors(N, m, k, seed=3, shift=float(N))
    At = torch.from_numpy(W.dense_from_factors(f)).to(DEV)
    op = hm.hm_dense_operator_create(At)
    t = hm.Tree(N, m)
    # r = 10 < k = 16: every block's rank saturates
    h = hm.hm_compress_hodlr(op, t, tol=1e-10, r=10, seed=2, prec=hm.HM_FP64)
    assert h.info["saturated"] > 0
    with pytest.raises(hm.HmError) as e:
        hm.hm_compress_hodlr(op, t, tol=1e-10, r=10, seed=2, prec=hm.HM_FP64, strict_rank=1)
    assert e.value.status == 5  # HM_ERANK_SATURATED
    # r above the rank: no saturation, strict mode passes
    h = hm.hm_compress_hodlr(op, t, tol=1e-10, r=k + 10, seed=2, prec=hm.HM_FP64, strict_rank=1)
    assert h.info["saturated"] == 0 and h.info["max_rank"] == k


def test_strict_rank_hbsid():
    N, m = 1024, 64
    At = torch.from_numpy(W.log_kernel(N).astype(np.float64)).to(DEV)
    op = hm.hm_dense_operator_create(At)
    t = hm.Tree(N, m)
    # tol 1e-12 needs ranks above 8 on the log kernel
    h = hm.hm_compress_hbs(op, t, tol=1e-12, r=8, seed=2, prec=hm.HM_FP64, hbs_id=1)
    assert h.info["saturated"] > 0
    with pytest.raises(hm.HmError) as e:
        hm.hm_compress_hbs(op, t, tol=1e-12, r=8, seed=2, prec=hm.HM_FP64, hbs_id=1,
                           strict_rank=1)
    assert e.value.status == 5
