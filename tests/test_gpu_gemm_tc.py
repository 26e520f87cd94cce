"""The tensor-core sampling GEMM (tcgen05, three-way BF16 split) against an FP64
product and against the CUDA-core engine, through the C ABI."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
DEV = "cuda:0"


def run(A32, X, trans, cuda_cores=False):
    N, c = X.shape
    At = torch.from_numpy(A32).to(DEV)
    op = hm.hm_dense_operator_create(At, cuda_cores=cuda_cores)
    Xd = torch.from_numpy(np.ascontiguousarray(X.T.astype(np.float32))).to(DEV)
    Y = torch.full((c, N), float("nan"), device=DEV)
    hm.hm_dense_apply(op, trans, Xd, Y)
    torch.cuda.synchronize()
    return Y.double().cpu().numpy().T


@pytest.mark.parametrize("N,c", [(1000, 37), (512, 64), (1536, 60), (777, 130)])
@pytest.mark.parametrize("trans", [0, 1])
def test_tc_gemm_bf16_exact_x(N, c, trans):
    """X with BF16 values (three products), half of its rows zero."""
    rng = np.random.default_rng(N + c + trans)
    A = rng.standard_normal((N, N)).astype(np.float32)
    X = rng.standard_normal((N, c)).astype(np.float32)
    X = torch.from_numpy(X).to(torch.bfloat16).to(torch.float32).numpy()
    X[: N // 2] = 0.0
    got = run(A, X, trans)
    want = (A.astype(np.float64).T if trans else A.astype(np.float64)) @ X.astype(np.float64)
    assert np.all(np.isfinite(got))
    err = np.abs(got - want) / np.sqrt(np.sum(want ** 2, axis=0, keepdims=True) / N)
    assert err.max() < 2e-6, err.max()


@pytest.mark.parametrize("N,c", [(1000, 37), (2048, 64)])
@pytest.mark.parametrize("trans", [0, 1])
def test_tc_gemm_general_x_matches_cuda_cores(N, c, trans):
    """General FP32 X (six products) against FP64 and the CUDA-core engine."""
    rng = np.random.default_rng(7 * N + c)
    A = rng.standard_normal((N, N)).astype(np.float32)
    Q, _ = np.linalg.qr(rng.standard_normal((N, c)))
    X = Q.astype(np.float32)
    got = run(A, X, trans)
    ref = run(A, X, trans, cuda_cores=True)
    want = (A.astype(np.float64).T if trans else A.astype(np.float64)) @ X.astype(np.float64)
    scale = np.sqrt(np.sum(want ** 2, axis=0, keepdims=True) / N)
    e_tc = (np.abs(got - want) / scale).max()
    e_cc = (np.abs(ref - want) / scale).max()
    print(f"N={N} c={c} trans={trans}: tensor-core {e_tc:.2e}, CUDA-core {e_cc:.2e}")
    assert e_tc < 2e-6


def test_tc_gemm_zero_block_and_identity_probe():
    N = 640
    rng = np.random.default_rng(3)
    A = rng.standard_normal((N, N)).astype(np.float32)
    X = np.zeros((N, 64), np.float32)
    assert np.all(run(A, X, 0) == 0.0)
    # identity probe with 64-row leaves: Y(i, c) = sum over leaves of A(i, s_leaf + c)
    for s in range(0, N, 64):
        X[s:s + 64] = np.eye(64, dtype=np.float32)
    got = run(A, X, 0)
    want = sum(A[:, s:s + 64].astype(np.float64) for s in range(0, N, 64))
    assert np.abs(got - want).max() < 1e-5
