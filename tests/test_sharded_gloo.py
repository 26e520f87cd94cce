"""The row-sharded black box on a world of two ranks (gloo on the CPU): its
products equal the dense ones, and a compression driven through it on every
rank equals the single-process compression (the FP64 oracle's, Fig. "Randomized
compression of a HODLR matrix"), with identical results on both ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W

hm = pytest.importorskip("paper_1503_07152_gb300")
from paper_1503_07152_gb300 import sharded  # noqa: E402

N, M, K = 512, 32, 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import hodlr as ohodlr
    from oracle.tree import build_tree
    A = W.dense_from_factors(W.synthetic_hodlr_factors(N, M, K, seed=7, shift=float(N)))
    ranges = sharded.tree_row_ranges(N, M, world)
    r0, r1 = ranges[rank]
    op = sharded.RowShardedOperator(torch.from_numpy(A[r0:r1].copy()), N, ranges)
    X = torch.from_numpy(np.random.default_rng(1).standard_normal((6, N)))
    for trans in (0, 1):
        Y = op.apply(X, trans).numpy().T
        want = (A.T if trans else A) @ X.numpy().T
        assert np.max(np.abs(Y - want)) <= 1e-12 * np.max(np.abs(want))

    def apply_fn(Xn, transpose):
        return op.apply(torch.from_numpy(np.ascontiguousarray(Xn.T)), int(transpose)).numpy().T
    h = ohodlr.compress(apply_fn, build_tree(N, M), r=K + 10, k=K, seed=2)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), ohodlr.dense(h))
    dist.destroy_process_group()


def test_row_ranges_follow_the_tree():
    t = hm.Tree(1000, 64)
    rr = sharded.tree_row_ranges(1000, 64, 4)
    assert rr == [(s, s + z) for s, z in (t.node(4 + p) for p in range(4))]
    assert rr[0][0] == 0 and rr[-1][1] == 1000
    assert all(rr[i][1] == rr[i + 1][0] for i in range(3))
    with pytest.raises(ValueError):
        sharded.tree_row_ranges(1000, 64, 3)


def test_two_rank_sharded_compression_matches_single_process(tmp_path):
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    from oracle import hodlr as ohodlr
    from oracle.tree import build_tree
    A = W.dense_from_factors(W.synthetic_hodlr_factors(N, M, K, seed=7, shift=float(N)))
    ref = ohodlr.dense(ohodlr.compress(ohodlr.dense_apply_fn(A), build_tree(N, M), r=K + 10, k=K,
                                       seed=2))
    d0, d1 = np.load(tmp_path / "rank0.npy"), np.load(tmp_path / "rank1.npy")
    assert np.array_equal(d0, d1)
    assert np.linalg.norm(d0 - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.linalg.norm(d0 - A) <= 1e-12 * np.linalg.norm(A)
