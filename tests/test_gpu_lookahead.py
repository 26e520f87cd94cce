"""Look-ahead sampling (hm_opts.lookahead): the A-side test matrix of every level
is a fresh Gaussian block, so the compression applies the black box to the next
level's block on a second stream while it factors the current level's samples.
The products, the kernels and the order of every reduction are unchanged, so a
compression with look-ahead must equal the one without it bit for bit: through
the library's black boxes (dense tensor-core split GEMM, matrix-free log kernel,
BF16x3 FP32 GEMM) and through a user callback that honours the stream argument,
for HODLR and HBS-ID handles."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
DEV = "cuda:0"


def dense_of(h, N, dtype=torch.float64, stream=None):
    out = torch.empty((N, N), device=DEV, dtype=dtype)
    hm.hm_reconstruct_block(h, 0, N, 0, N, out, stream=stream)
    torch.cuda.synchronize()
    return out


def _log_kernel_box(kind, N):
    if kind == "matrix_free":
        return hm.hm_log_kernel_operator_create(N), hm.HM_A32, torch.float64
    A = torch.empty((N, N), device=DEV, dtype=torch.float32)
    hm.hm_gen_log_kernel(A)
    if kind == "split_tc":
        return hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True), hm.HM_A32, \
            torch.float64
    return hm.hm_dense_operator_create(A), hm.HM_MIXED, torch.float32  # BF16x3 on tensor cores


@pytest.mark.parametrize("fmt", ["hodlr", "hbsid"])
@pytest.mark.parametrize("kind", ["split_tc", "matrix_free", "bf16x3"])
def test_lookahead_equals_in_order_sampling(fmt, kind):
    N, m = 8192, 256
    op, prec, dt = _log_kernel_box(kind, N)
    t = hm.Tree(N, m)
    comp = hm.hm_compress_hodlr if fmt == "hodlr" else hm.hm_compress_hbs
    kw = dict(tol=1e-7, r=60, prec=prec)
    h_off = comp(op, t, lookahead=-1, **kw)
    h_on = comp(op, t, lookahead=0, **kw)  # on: the library's own black box
    assert torch.equal(dense_of(h_off, N, dt), dense_of(h_on, N, dt))
    for key in ("max_rank", "min_rank", "saturated", "cols_A", "cols_At"):
        assert h_on.info[key] == h_off.info[key], key
    if fmt == "hbsid":
        for node in (2, 3, 9, 2 * t.levels + 1):
            for side in (0, 1):
                assert np.array_equal(hm.hm_skeleton(h_on, node, side),
                                      hm.hm_skeleton(h_off, node, side))


def test_lookahead_waits_for_the_callers_stream():
    """The operator is generated on a side stream and compressed on that stream
    at once: both of the compression's own streams must start after the
    generator, and the reconstruction queued on the caller's stream after the
    compression's end."""
    N, m = 8192, 256
    s = torch.cuda.Stream()
    A = torch.empty((N, N), device=DEV, dtype=torch.float32)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        A.fill_(float("nan"))
        hm.hm_gen_log_kernel(A, stream=s)
        op = hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True)
        t = hm.Tree(N, m)
        h_on = hm.hm_compress_hbs(op, t, tol=1e-7, r=60, prec=hm.HM_A32, lookahead=0, stream=s)
        got = dense_of(h_on, N, stream=s)
    h_off = hm.hm_compress_hbs(op, t, tol=1e-7, r=60, prec=hm.HM_A32, lookahead=-1)
    assert torch.equal(got, dense_of(h_off, N))


@pytest.mark.parametrize("fmt", ["hodlr", "hbsid"])
def test_lookahead_user_callback(fmt):
    """A user black box (torch products on the stream it is given) with
    lookahead = 1: called on two streams with calls in flight on both."""
    from paper_1503_07152_gb300.sharded import _DeviceBlock
    N, m, k = 2048, 64, 10
    if fmt == "hodlr":  # exact-rank HODLR input
        A = W.dense_from_factors(W.synthetic_hodlr_factors(N, m, k, seed=11, shift=float(N)))
    else:  # the log kernel: nested bases
        A = W.log_kernel(N).astype(np.float64)
    Ad = torch.from_numpy(A).to(DEV)
    calls = set()

    def fn(trans, X, ldx, Y, ldy, ncols, stream):
        calls.add(int(stream or 0))
        xs = torch.as_tensor(_DeviceBlock(X, ncols, ldx), device=DEV)[:, :N]
        ys = torch.as_tensor(_DeviceBlock(Y, ncols, ldy), device=DEV)[:, :N]
        strm = torch.cuda.ExternalStream(stream, device=DEV) if stream else \
            torch.cuda.default_stream(DEV)
        with torch.cuda.stream(strm):
            ys.copy_(xs @ (Ad if trans else Ad.T))  # rows of ys: columns of op(A) X
        return 0

    op = hm.callback_operator(N, fn)
    t = hm.Tree(N, m)
    comp = hm.hm_compress_hodlr if fmt == "hodlr" else hm.hm_compress_hbs
    kw = dict(k=k, p=10, prec=hm.HM_FP64) if fmt == "hodlr" else \
        dict(tol=1e-7, r=40, prec=hm.HM_FP64)
    h_off = comp(op, t, lookahead=-1, **kw)
    calls_off = set(calls)
    calls.clear()
    h_on = comp(op, t, lookahead=1, **kw)
    assert len(calls_off) == 1 and len(calls) == 2  # in order: one stream; look-ahead: two
    # the products are the caller's cuBLAS calls, deterministic for equal shapes
    assert torch.equal(dense_of(h_off, N), dense_of(h_on, N))
    if fmt == "hodlr":  # exact-rank HODLR input: recovered to rounding
        assert np.linalg.norm(dense_of(h_on, N).cpu().numpy().T - A) / np.linalg.norm(A) < 1e-12
