"""The row-sharded black box driving the library's compression on the GPU: the
callback path (device blocks wrapped as tensors, products on the library's
stream, collectives of a one-rank NCCL group) gives the same compression as the
library's dense FP64 operator.  The multi-rank products are covered on the CPU
(tests/test_sharded_gloo.py); every call here takes one GPU."""
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist

import workloads as W

pytestmark = pytest.mark.gpu
hm = pytest.importorskip("paper_1503_07152_gb300")
from paper_1503_07152_gb300 import sharded  # noqa: E402

DEV = "cuda:0"


def test_sharded_black_box_compression_on_one_rank():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        N, m, k = 1024, 64, 8
        A = W.dense_from_factors(W.synthetic_hodlr_factors(N, m, k, seed=9, shift=float(N)))
        At = torch.from_numpy(A).to(DEV)
        ranges = sharded.tree_row_ranges(N, m, 1)
        op = sharded.RowShardedOperator(At, N, ranges).black_box()
        t = hm.Tree(N, m)
        h = hm.hm_compress_hodlr(op, t, k=k, p=10, seed=2, prec=hm.HM_FP64)
        hd = hm.hm_compress_hodlr(hm.hm_dense_operator_create(At), t, k=k, p=10, seed=2,
                                  prec=hm.HM_FP64)
        out = [torch.empty((N, N), device=DEV, dtype=torch.float64) for _ in range(2)]
        hm.hm_reconstruct_block(h, 0, N, 0, N, out[0])
        hm.hm_reconstruct_block(hd, 0, N, 0, N, out[1])
        torch.cuda.synchronize()
        nA = np.linalg.norm(A)
        assert float((out[0] - out[1]).norm()) <= 1e-12 * nA
        assert np.linalg.norm(out[0].cpu().numpy().T - A) <= 1e-12 * nA
    finally:
        dist.destroy_process_group()
