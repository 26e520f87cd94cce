"""Row-sharded black box: one operator held as row blocks on the ranks of a
torch.distributed process group, for operators too large for one device (the
black-box products dominate the compression, Sec. 5's closing remarks).

Rank p holds A(I_p, :), where I_p is the index range of node 2^g + p of the
compression tree on level g = log2(world size): the row blocks follow the tree,
so each rank's rows are whole subtrees.  Products:
  Y = A X:    every rank forms Y(I_p, :) = A(I_p, :) X and the blocks are
              all-gathered (every rank ends with the whole Y);
  Y = A^T X:  every rank forms A(I_p, :)^T X(I_p, :) and the partial sums are
              all-reduced.
Every rank then runs the same (replicated) compression on identical samples, so
all ranks hold the same handle.  The local products are plain torch matmuls on
the rank's device; the communication is the process group's (NCCL across GPUs,
gloo on the CPU).
"""
from __future__ import annotations

import ctypes as C

import torch
import torch.distributed as dist

from . import _lib


def tree_row_ranges(n: int, leaf_size: int, world: int) -> list:
    """(start, stop) of the rows of each rank: the nodes of the tree level with
    `world` nodes (world must be a power of two no larger than the leaf count)."""
    if world < 1 or world & (world - 1):
        raise ValueError("the world size must be a power of two")
    t = _lib.Tree(n, leaf_size)
    g = world.bit_length() - 1
    if g > t.levels:
        raise ValueError("more ranks than leaves")
    out = []
    for p in range(world):
        s, z = t.node((1 << g) + p)
        out.append((s, s + z))
    return out


class RowShardedOperator:
    """A(I_p, :) on this rank; apply() gives op(A) X on every rank."""

    def __init__(self, A_local: torch.Tensor, n: int, ranges: list, group=None):
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        if len(ranges) != self.world:
            raise ValueError("one row range per rank")
        r0, r1 = ranges[self.rank]
        if A_local.shape != (r1 - r0, n):
            raise ValueError("A_local must hold this rank's rows, all n columns")
        self.A, self.n, self.ranges = A_local, n, ranges
        self.rows_max = max(b - a for a, b in ranges)

    def apply(self, X: torch.Tensor, trans: int) -> torch.Tensor:
        """X: (ncols, n) tensor (the column-major n x ncols block); returns (ncols, n)."""
        r0, r1 = self.ranges[self.rank]
        if not trans:
            loc = X @ self.A.T  # (ncols, rows of this rank)
            pad = torch.zeros((X.shape[0], self.rows_max), dtype=X.dtype, device=X.device)
            pad[:, : r1 - r0] = loc
            parts = [torch.empty_like(pad) for _ in range(self.world)]
            dist.all_gather(parts, pad, group=self.group)
            Y = torch.empty((X.shape[0], self.n), dtype=X.dtype, device=X.device)
            for (a, b), part in zip(self.ranges, parts):
                Y[:, a:b] = part[:, : b - a]
            return Y
        Y = X[:, r0:r1] @ self.A  # (ncols, n) partial sum of A^T X
        dist.all_reduce(Y, group=self.group)
        return Y

    def black_box(self) -> "_lib.Operator":
        """The library black box (double blocks on this rank's CUDA device) for
        hm_compress_*: the callback wraps the library's device blocks as tensors
        and runs apply() on the library's stream."""
        n = self.n
        dev = self.A.device

        def fn(trans, X, ldx, Y, ldy, ncols, stream):
            xs = torch.as_tensor(_DeviceBlock(X, ncols, ldx), device=dev)[:, :n]
            ys = torch.as_tensor(_DeviceBlock(Y, ncols, ldy), device=dev)[:, :n]
            # a null stream is the legacy default stream, torch's default stream
            strm = (torch.cuda.ExternalStream(stream, device=dev) if stream
                    else torch.cuda.default_stream(dev))
            with torch.cuda.stream(strm):
                ys.copy_(self.apply(xs, trans))
            return 0
        return _lib.callback_operator(n, fn)


class _DeviceBlock:
    """__cuda_array_interface__ view of a column-major double block."""

    def __init__(self, ptr, ncols, ld):
        addr = ptr if isinstance(ptr, int) else C.cast(ptr, C.c_void_p).value
        self.__cuda_array_interface__ = {"shape": (int(ncols), int(ld)), "typestr": "<f8",
                                         "data": (int(addr), False), "version": 3,
                                         "strides": None}
