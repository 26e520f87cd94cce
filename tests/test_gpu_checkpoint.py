"""Checkpoint of compressed handles (hm_save / hm_load) through the C ABI: the
loaded handle reproduces the saved one's applies bit for bit; damaged files are
rejected."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
DEV = "cuda:0"


def _apply_both(h, N, dtype, seed=0):
    X = torch.from_numpy(np.random.default_rng(seed).standard_normal((4, N))).to(DEV, dtype)
    out = []
    for trans in (0, 1):
        Y = torch.empty_like(X)
        hm.hm_apply(h, trans, X, Y)
        out.append(Y)
    torch.cuda.synchronize()
    return [y.cpu().numpy() for y in out]


@pytest.mark.parametrize("kind", ["hodlr_fp64", "hbsid_a32", "hodlr_mixed"])
def test_save_load_roundtrip(tmp_path, kind):
    if kind == "hodlr_fp64":
        N, m = 1000, 64
        f = W.synthetic_hodlr_factors(N, m, 7, seed=1, shift=float(N))
        At = torch.from_numpy(W.dense_from_factors(f)).to(DEV)
        h = hm.hm_compress_hodlr(hm.hm_dense_operator_create(At), hm.Tree(N, m), k=7, p=10,
                                 prec=hm.HM_FP64)
        dtype = torch.float64
    elif kind == "hbsid_a32":
        N, m = 2048, 128
        At = torch.from_numpy(W.log_kernel(N)).to(DEV)
        op = hm.hm_dense_operator_create(At, fp64_blocks=True, tensor_cores=True)
        h = hm.hm_compress_hbs(op, hm.Tree(N, m), tol=1e-7, r=40, prec=hm.HM_A32, hbs_id=1)
        dtype = torch.float64
    else:
        N, m = 1500, 64
        At = torch.from_numpy(W.log_kernel(N)).to(DEV)
        h = hm.hm_compress_hodlr(hm.hm_dense_operator_create(At), hm.Tree(N, m), tol=1e-6, r=30,
                                 prec=hm.HM_MIXED)
        dtype = torch.float32
    path = str(tmp_path / f"{kind}.hm")
    hm.hm_save(h, path)
    g = hm.hm_load(path)
    assert g.info == h.info
    for a, b in zip(_apply_both(h, N, dtype), _apply_both(g, N, dtype)):
        assert np.array_equal(a, b)
    if kind == "hbsid_a32":
        for node in (2, 3, 17):
            assert hm.hm_skeleton(g, node, 0) == hm.hm_skeleton(h, node, 0)
    # a flipped payload byte and a truncated file are rejected
    raw = bytearray(open(path, "rb").read())
    raw[-5] ^= 0x40
    bad = str(tmp_path / "bad.hm")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(hm.HmError) as e:
        hm.hm_load(bad)
    assert e.value.status == 1
    open(bad, "wb").write(bytes(raw[: len(raw) // 2]))
    with pytest.raises(hm.HmError) as e:
        hm.hm_load(bad)
    assert e.value.status == 1


def test_loaded_hodlr_can_be_factorized(tmp_path):
    N, m = 1024, 64
    f = W.synthetic_hodlr_factors(N, m, 6, seed=2, shift=float(N))
    A = W.dense_from_factors(f)
    h = hm.hm_compress_hodlr(hm.hm_dense_operator_create(torch.from_numpy(A).to(DEV)),
                             hm.Tree(N, m), k=6, p=10, prec=hm.HM_FP64)
    path = str(tmp_path / "f.hm")
    hm.hm_save(h, path)
    g = hm.hm_load(path)
    hm.hm_hodlr_factorize(g)
    b = torch.ones((1, N), device=DEV, dtype=torch.float64)
    x = torch.empty_like(b)
    hm.hm_solve(g, 0, b, x)
    torch.cuda.synchronize()
    assert np.linalg.norm(A @ x.cpu().numpy()[0] - 1.0) <= 1e-10 * np.sqrt(N)
