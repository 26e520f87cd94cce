"""The hand-written adjoint of the factored HODLR apply (FP32 kernels, through
torch.autograd) against FP64 central finite differences of the loss
||H x - b||^2 at N = 4096 (k = 32, leaves of 256 points, the shape of the
differentiation workload at a size where differences are cheap).

The loss is quadratic in every single entry of x, U, V and D, so a central
difference is exact up to rounding: the comparison measures the FP32 adjoint
itself.  Sampled entries of every argument, compared as one vector per
argument."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import grad as ograd

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
DEV = "cuda:0"


def _loss64(f, x, b):
    return ograd.loss(f, x, b)


def test_adjoint_against_central_differences():
    N, m, k = 4096, 256, 32
    f = W.synthetic_hodlr_factors(N, m, k, seed=5, shift=0.0, dtype=np.float32)
    L = f["L"]
    rng = np.random.default_rng(6)
    x = rng.standard_normal(N).astype(np.float32)
    b = rng.standard_normal(N).astype(np.float32)
    t = hm.Tree(N, m)
    U = torch.from_numpy(np.stack([np.ascontiguousarray(f["U"][j].T) for j in range(1, L + 1)])).to(DEV).requires_grad_()
    V = torch.from_numpy(np.stack([np.ascontiguousarray(f["V"][j].T) for j in range(1, L + 1)])).to(DEV).requires_grad_()
    D = torch.from_numpy(np.stack([d.T.copy() for d in f["D"]])).to(DEV).requires_grad_()
    xd = torch.from_numpy(x).to(DEV).requires_grad_()
    y = hm.HodlrApply.apply(xd, U, V, D, t, k)
    loss = ((y - torch.from_numpy(b).to(DEV)) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    # FP64 copies of the same (FP32-valued) factors for the differences
    f64 = dict(f)
    f64["U"] = [None] + [f["U"][j].astype(np.float64) for j in range(1, L + 1)]
    f64["V"] = [None] + [f["V"][j].astype(np.float64) for j in range(1, L + 1)]
    f64["D"] = [d.astype(np.float64) for d in f["D"]]
    x64, b64 = x.astype(np.float64), b.astype(np.float64)
    h = 1e-3
    pick = np.random.default_rng(7)
    worst = {}

    def fd(setter):
        setter(+h)
        lp = _loss64(f64, x64, b64)
        setter(-2 * h)
        lm = _loss64(f64, x64, b64)
        setter(+h)
        return (lp - lm) / (2 * h)

    # x
    g_gpu, g_fd = [], []
    for i in pick.choice(N, 12, replace=False):
        def s(d, i=i):
            x64[i] += d
        g_fd.append(fd(s))
        g_gpu.append(float(xd.grad[i]))
    worst["x"] = np.linalg.norm(np.array(g_gpu) - g_fd) / np.linalg.norm(g_fd)
    # U, V (level j, row i, column c), stored as (level, column, row) on the device
    for name, arr, grad in (("U", f64["U"], U.grad), ("V", f64["V"], V.grad)):
        g_gpu, g_fd = [], []
        for _ in range(12):
            j, i, c = int(pick.integers(1, L + 1)), int(pick.integers(N)), int(pick.integers(k))

            def s(d, j=j, i=i, c=c, arr=arr):
                arr[j][i, c] += d
            g_fd.append(fd(s))
            g_gpu.append(float(grad[j - 1, c, i]))
        worst[name] = np.linalg.norm(np.array(g_gpu) - g_fd) / np.linalg.norm(g_fd)
    # D (leaf l, row i, column c), stored column-major per leaf
    g_gpu, g_fd = [], []
    for _ in range(12):
        l, i, c = int(pick.integers(len(f64["D"]))), int(pick.integers(m)), int(pick.integers(m))

        def s(d, l=l, i=i, c=c):
            f64["D"][l][i, c] += d
        g_fd.append(fd(s))
        g_gpu.append(float(D.grad[l, c, i]))
    worst["D"] = np.linalg.norm(np.array(g_gpu) - g_fd) / np.linalg.norm(g_fd)
    print("adjoint vs central differences (relative, per argument): "
          + ", ".join(f"{k_}: {v:.2e}" for k_, v in worst.items()))
    for name, v in worst.items():  # measured 1.9e-7 .. 3.8e-7 (FP32 rounding of the kernels)
        assert v < 1e-6, (name, v)
