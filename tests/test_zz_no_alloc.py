"""hm_hodlr_factored_apply_noalloc (scratch in a static device buffer) against
hm_hodlr_factored_apply, through the C ABI.  Collected last on purpose: it must
give the same results after everything else has run in the process."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
DEV = "cuda:0"


def factors(N, m, k, seed):
    f = W.synthetic_hodlr_factors(N, m, k, seed=seed, shift=0.0, dtype=np.float32)
    L = f["L"]
    nmax = max(d.shape[0] for d in f["D"])
    U = torch.from_numpy(np.stack([np.ascontiguousarray(f["U"][j].T) for j in range(1, L + 1)])).to(DEV)
    V = torch.from_numpy(np.stack([np.ascontiguousarray(f["V"][j].T) for j in range(1, L + 1)])).to(DEV)
    Dp = np.zeros((len(f["D"]), nmax, nmax), np.float32)
    for i, d in enumerate(f["D"]):
        Dp[i, : d.shape[0], : d.shape[0]] = d.T
    return U, V, torch.from_numpy(Dp).to(DEV)


@pytest.mark.parametrize("N,m,k", [(4096, 128, 16), (3000, 100, 7), (65536, 256, 32)])
@pytest.mark.parametrize("trans", [0, 1])
def test_noalloc_matches_allocating_apply(N, m, k, trans):
    t = hm.Tree(N, m)
    U, V, D = factors(N, m, k, seed=N + k)
    x = torch.randn(N, device=DEV, generator=torch.Generator(DEV).manual_seed(k))
    want = torch.empty_like(x)
    hm.hm_hodlr_factored_apply(t, k, U, V, D, x, want, trans=trans)  # also uploads the tree
    for _ in range(2):  # two calls in a row reuse the same static scratch
        y = torch.full_like(x, float("nan"))
        hm.hm_hodlr_factored_apply_noalloc(t, k, U, V, D, x, y, trans=trans)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        assert torch.linalg.norm(y - want) <= 1e-6 * torch.linalg.norm(want)


def test_noalloc_needs_uploaded_tree():
    t = hm.Tree(2048, 64)
    U, V, D = factors(2048, 64, 4, seed=1)
    x = torch.randn(2048, device=DEV)
    y = torch.empty_like(x)
    with pytest.raises(hm.HmError, match="not on the device"):
        hm.hm_hodlr_factored_apply_noalloc(t, 4, U, V, D, x, y)


def test_noalloc_rejects_oversized_scratch():
    # N = 2^20 with 64-point leaves and k = 64 needs about 23 MB of scratch
    t = hm.Tree(1 << 20, 64)
    dummy = torch.empty(1, device=DEV)
    with pytest.raises(hm.HmError, match="static buffer holds"):
        hm.hm_hodlr_factored_apply_noalloc(t, 64, dummy, dummy, dummy, dummy, dummy)
