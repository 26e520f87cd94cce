"""ctypes marshalling for libhm.so (argument checks and pointer plumbing only)."""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libhm.so")

HM_FP64, HM_MIXED, HM_A32 = 0, 1, 2
HM_FORMAT_HODLR, HM_FORMAT_HBS, HM_FORMAT_HBSID = 0, 1, 2
_STATUS = {0: "HM_OK", 1: "HM_EINVAL", 2: "HM_ENOMEM", 3: "HM_ECUDA", 4: "HM_ECALLBACK",
           5: "HM_ERANK_SATURATED", 6: "HM_ENONFINITE", 7: "HM_ETIMEOUT", 8: "HM_EUNSUPPORTED"}

if not os.path.exists(library_path):
    raise ImportError(
        f"{library_path} is missing: build it with `python paper_1503_07152_gb300/build.py` "
        "(or __graft_entry__.build()); there is no fallback path")
lib = C.CDLL(library_path)

APPLY_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_int64,
                       C.c_void_p, C.c_int64, C.c_void_p)


class _Operator(C.Structure):
    _fields_ = [("apply", APPLY_FN), ("ctx", C.c_void_p), ("n", C.c_int64)]


class Opts(C.Structure):
    _fields_ = [("mode_tol", C.c_int32), ("k", C.c_int32), ("tol", C.c_double), ("p", C.c_int32),
                ("r", C.c_int32), ("leaf_size", C.c_int32), ("seed", C.c_uint64),
                ("prec", C.c_int32), ("hbs_id", C.c_int32), ("strict_rank", C.c_int32),
                ("lookahead", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("format", C.c_int32), ("prec", C.c_int32), ("n", C.c_int64),
                ("levels", C.c_int32), ("r", C.c_int32), ("max_rank", C.c_int32),
                ("min_rank", C.c_int32), ("saturated", C.c_int32), ("cols_A", C.c_int64),
                ("cols_At", C.c_int64), ("bytes", C.c_int64), ("eps_abs", C.c_double),
                ("t_compress_ms", C.c_double), ("t_blackbox_ms", C.c_double),
                ("launches", C.c_int32)]


class _Phase(C.Structure):
    _fields_ = [("level", C.c_int32), ("side", C.c_int32), ("phase", C.c_int32), ("ms", C.c_double)]


PHASES = ["sample", "peel", "tsqr", "svd", "orth", "bases", "id"]

_P = C.c_void_p
_sig = {
    "hm_tree_create": ([C.c_int64, C.c_int32, C.POINTER(_P)], C.c_int),
    "hm_tree_destroy": ([_P], None),
    "hm_tree_levels": ([_P], C.c_int32),
    "hm_tree_node": ([_P, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "hm_dense_operator_create": ([_P, C.c_int64, C.c_int64, C.c_int32, C.POINTER(_Operator)], C.c_int),
    "hm_dense_operator_destroy": ([C.POINTER(_Operator)], None),
    "hm_dense_apply": ([C.POINTER(_Operator), C.c_int, C.c_int64, _P, C.c_int64, _P, C.c_int64, _P], C.c_int),
    "hm_compress_hodlr": ([C.POINTER(_Operator), _P, C.POINTER(Opts), _P, C.POINTER(_P)], C.c_int),
    "hm_compress_hbs": ([C.POINTER(_Operator), _P, C.POINTER(Opts), _P, C.POINTER(_P)], C.c_int),
    "hm_compress_batched": ([C.c_int32, C.POINTER(_Operator), C.POINTER(_P), C.POINTER(Opts), C.c_int32,
                             C.c_int32, _P, C.POINTER(_P)], C.c_int),
    "hm_tune_batched": ([C.c_int32, C.POINTER(_Operator), C.POINTER(_P), C.POINTER(Opts), C.c_int32,
                         C.POINTER(C.c_int32), C.c_int32, _P, C.POINTER(C.c_int32),
                         C.POINTER(C.c_double)], C.c_int),
    "hm_apply": ([_P, C.c_int, C.c_int64, _P, C.c_int64, _P, C.c_int64, _P], C.c_int),
    "hm_apply_host": ([_P, C.c_int, C.c_int64, _P, C.c_int64, _P, C.c_int64, _P], C.c_int),
    "hm_reconstruct_block": ([_P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, _P, C.c_int64, _P], C.c_int),
    "hm_rel_frob_error": ([_P, _P, C.c_int64, C.c_int32, C.POINTER(C.c_double), _P], C.c_int),
    "hm_info": ([_P, C.POINTER(_Info)], C.c_int),
    "hm_node_rank": ([_P, C.c_int64, C.POINTER(C.c_int32)], C.c_int),
    "hm_destroy": ([_P], None),
    "hm_set_profiling": ([C.c_int32], C.c_int),
    "hm_profile": ([_P, C.POINTER(_Phase), C.c_int32, C.POINTER(C.c_int32)], C.c_int),
    "hm_hodlr_factorize": ([_P, _P], C.c_int),
    "hm_save": ([_P, C.c_char_p], C.c_int),
    "hm_load": ([C.c_char_p, _P, C.POINTER(_P)], C.c_int),
    "hm_product_operator_create": ([C.c_int32, C.POINTER(_P), C.POINTER(C.c_int32), C.c_double,
                                    C.c_double, C.POINTER(_Operator)], C.c_int),
    "hm_product_operator_destroy": ([C.POINTER(_Operator)], None),
    "hm_solve": ([_P, C.c_int, C.c_int64, _P, C.c_int64, _P, C.c_int64, _P], C.c_int),
    "hm_skeleton": ([_P, C.c_int64, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int32)], C.c_int),
    "hm_hodlr_factored_apply": ([_P, C.c_int32, _P, _P, _P, C.c_int, _P, _P, _P], C.c_int),
    "hm_hodlr_factored_apply_noalloc": ([_P, C.c_int32, _P, _P, _P, C.c_int, _P, _P, _P], C.c_int),
    "hm_hodlr_factored_adjoint": ([_P, C.c_int32, _P, _P, _P, _P, _P, C.c_float, _P, _P, _P, _P, _P],
                                  C.c_int),
    "hm_hodlr_factored_loss_grad": ([_P, C.c_int32, _P, _P, _P, _P, _P, C.c_float, _P, _P, _P, _P,
                                     _P, _P, _P], C.c_int),
    "hm_gen_log_kernel": ([_P, C.c_int64, C.c_int64, _P], C.c_int),
    "hm_hodlr_export_level": ([_P, C.c_int32, _P, _P, _P], C.c_int),
    "hm_gaussian_test_matrix": ([_P, C.c_int32, C.c_int32, C.c_uint64, C.c_int32, _P, C.c_int64, _P],
                                C.c_int),
    "hm_dense_operator_check": ([C.POINTER(_Operator), _P], C.c_int),
    "hm_log_kernel_operator_create": ([C.c_int64, C.POINTER(_Operator)], C.c_int),
    "hm_log_kernel_entries": ([C.POINTER(_Operator), C.c_int64, C.c_int64, C.c_int64, C.c_int64, _P,
                               C.c_int64, _P], C.c_int),
    "hm_set_wait_limit": ([C.c_int64], C.c_int),
    "hm_last_error": ([], C.c_char_p),
    "hm_version": ([], C.c_char_p),
    "hm_launch_count": ([], C.c_int64),
}
for _name, (_args, _ret) in _sig.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _ret


class HmError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib.hm_last_error().decode()
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, where: str) -> None:
    if status != 0:
        raise HmError(status, where)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _colmajor(t: torch.Tensor, n: int, name: str):
    """(ptr, ld, ncols) of a column-major n x ncols view given as a (ncols, ld) row-major tensor."""
    if t.dim() != 2 or t.shape[1] < n or t.stride(1) != 1:
        raise ValueError(f"{name} must be a (ncols, ld >= n) tensor with unit inner stride "
                         "(the column-major n x ncols block)")
    return C.c_void_p(t.data_ptr()), t.stride(0), t.shape[0]


def hm_version() -> str:
    return lib.hm_version().decode()


def hm_launch_count() -> int:
    return int(lib.hm_launch_count())


class Tree:
    def __init__(self, n: int, leaf_size: int):
        self.ptr = C.c_void_p()
        _check(lib.hm_tree_create(n, leaf_size, C.byref(self.ptr)), "hm_tree_create")
        self.n, self.leaf_size = n, leaf_size
        self.levels = lib.hm_tree_levels(self.ptr)

    def node(self, node: int):
        s, z = C.c_int64(), C.c_int64()
        _check(lib.hm_tree_node(self.ptr, node, C.byref(s), C.byref(z)), "hm_tree_node")
        return s.value, z.value

    def __del__(self):
        if getattr(self, "ptr", None):
            lib.hm_tree_destroy(self.ptr)
            self.ptr = None


def hm_tree_create(n: int, leaf_size: int) -> Tree:
    return Tree(n, leaf_size)


class Operator:
    """A black box: the library's dense, matrix-free or product operator, or a Python callback."""

    def __init__(self, op: _Operator, keep=None, dense: bool = False, product: bool = False):
        self.op = op
        self.keep = keep
        self.dense = dense
        self.product = product

    @property
    def n(self):
        return self.op.n

    def __del__(self):
        if getattr(self, "dense", False) and self.op.ctx:
            lib.hm_dense_operator_destroy(C.byref(self.op))
        if getattr(self, "product", False) and self.op.ctx:
            lib.hm_product_operator_destroy(C.byref(self.op))


def hm_dense_operator_create(A: torch.Tensor, fp64_blocks: bool = False,
                             cuda_cores: bool = False, tensor_cores: bool | None = None) -> Operator:
    """Dense test operator over a row-major (n, lda) CUDA tensor.  float64 -> HM_FP64.
    float32 -> HM_MIXED (tensor-core engine by default; cuda_cores=True: CUDA-core
    engine), or with fp64_blocks=True HM_A32 (float matrix, double blocks: exact FP64
    products on the CUDA cores by default; tensor_cores=True: the exact-accumulation
    split on the tensor cores)."""
    if A.dim() != 2 or A.stride(1) != 1 or not A.is_cuda:
        raise ValueError("A must be a row-major 2-D CUDA tensor")
    dtype = {torch.float64: 0, torch.float32: 1}[A.dtype]
    if fp64_blocks:
        if dtype != 1:
            raise ValueError("fp64_blocks needs a float32 matrix")
        dtype = 4 if tensor_cores else 2
    elif cuda_cores and dtype == 1:
        dtype = 3
    op = _Operator()
    _check(lib.hm_dense_operator_create(_ptr(A), A.shape[0], A.stride(0), dtype, C.byref(op)),
           "hm_dense_operator_create")
    return Operator(op, keep=A, dense=True)


def callback_operator(n: int, fn) -> Operator:
    """Black box from a Python callable fn(trans, X_ptr, ldx, Y_ptr, ldy, ncols, stream) -> int."""
    def tramp(ctx, trans, nn, ncols, X, ldx, Y, ldy, stream):
        try:
            return int(fn(trans, X, ldx, Y, ldy, ncols, stream))
        except Exception:  # an exception must not cross the C boundary: report it, fail the call
            import sys
            import traceback
            traceback.print_exc(file=sys.stderr)
            return 99
    cb = APPLY_FN(tramp)
    op = _Operator(cb, None, n)
    return Operator(op, keep=cb)


def hm_log_kernel_operator_create(n: int) -> Operator:
    """Matrix-free log-kernel black box of n ellipse points (HM_A32, double blocks)."""
    op = _Operator()
    _check(lib.hm_log_kernel_operator_create(n, C.byref(op)), "hm_log_kernel_operator_create")
    return Operator(op, dense=True)


def hm_log_kernel_entries(op: Operator, r0: int, r1: int, c0: int, c1: int, out: torch.Tensor,
                          stream=None) -> None:
    """out: row-major float32 CUDA tensor of shape (r1 - r0, ld >= c1 - c0)."""
    if out.dtype != torch.float32 or out.dim() != 2 or out.stride(1) != 1:
        raise ValueError("out must be a row-major float32 CUDA tensor")
    _check(lib.hm_log_kernel_entries(C.byref(op.op), r0, r1, c0, c1, _ptr(out), out.stride(0),
                                     C.c_void_p(_stream(stream))), "hm_log_kernel_entries")


def hm_dense_operator_check(op: Operator, stream=None) -> None:
    """Raises HmError (HM_ETIMEOUT) if a bounded wait of the operator's GEMMs gave up."""
    _check(lib.hm_dense_operator_check(C.byref(op.op), C.c_void_p(_stream(stream))),
           "hm_dense_operator_check")


def hm_set_wait_limit(polls: int) -> None:
    """Poll limit of the tensor-core GEMMs' pipeline waits (<= 0: the default)."""
    _check(lib.hm_set_wait_limit(int(polls)), "hm_set_wait_limit")


def hm_dense_apply(op: Operator, trans: int, X: torch.Tensor, Y: torch.Tensor, stream=None):
    px, ldx, ncols = _colmajor(X, op.n, "X")
    py, ldy, _ = _colmajor(Y, op.n, "Y")
    _check(lib.hm_dense_apply(C.byref(op.op), trans, ncols, px, ldx, py, ldy, C.c_void_p(_stream(stream))),
           "hm_dense_apply")


class Handle:
    def __init__(self, ptr: C.c_void_p, keep=None):
        self.ptr = ptr
        self.keep = keep
        self.info = hm_info(self)

    def __del__(self):
        if getattr(self, "ptr", None):
            lib.hm_destroy(self.ptr)
            self.ptr = None


def _opts(r=None, k=None, p=10, tol=None, leaf_size=0, seed=2, prec=HM_MIXED, hbs_id=1,
          strict_rank=0, lookahead=0) -> Opts:
    o = Opts()
    if tol is not None:
        o.mode_tol, o.tol, o.r = 1, float(tol), int(r if r is not None else 60)
    else:
        o.mode_tol, o.k, o.p = 0, int(k), int(p)
        o.r = int(k) + int(p)
    o.leaf_size, o.seed, o.prec, o.hbs_id, o.strict_rank = leaf_size, seed, prec, hbs_id, strict_rank
    o.lookahead = lookahead
    return o


def hm_compress_hodlr(op: Operator, tree: Tree, stream=None, **kw) -> Handle:
    o = _opts(**kw)
    h = C.c_void_p()
    _check(lib.hm_compress_hodlr(C.byref(op.op), tree.ptr, C.byref(o), C.c_void_p(_stream(stream)),
                                 C.byref(h)), "hm_compress_hodlr")
    return Handle(h, keep=(tree,))


def hm_compress_hbs(op: Operator, tree: Tree, stream=None, **kw) -> Handle:
    o = _opts(**kw)
    h = C.c_void_p()
    _check(lib.hm_compress_hbs(C.byref(op.op), tree.ptr, C.byref(o), C.c_void_p(_stream(stream)),
                               C.byref(h)), "hm_compress_hbs")
    return Handle(h, keep=(tree,))


def hm_compress_batched(ops: list, trees: list, fmt: str = "hodlr", opts: list | None = None,
                        max_concurrency: int = 0, stream=None) -> list:
    """Compress independent operators in one call; opts: one dict of hm_compress_* keywords
    per operator.  Returns one handle per operator."""
    n = len(ops)
    if len(trees) != n or (opts is not None and len(opts) != n):
        raise ValueError("ops, trees and opts must have the same length")
    opts = opts or [{} for _ in range(n)]
    ops_arr = (_Operator * n)(*[o.op for o in ops])
    trees_arr = (_P * n)(*[t.ptr for t in trees])
    opts_arr = (Opts * n)(*[_opts(**kw) for kw in opts])
    outs = (_P * n)()
    fmt_id = {"hodlr": HM_FORMAT_HODLR, "hbsid": HM_FORMAT_HBSID}[fmt]
    _check(lib.hm_compress_batched(n, ops_arr, trees_arr, opts_arr, fmt_id, max_concurrency,
                                   C.c_void_p(_stream(stream)), outs), "hm_compress_batched")
    return [Handle(C.c_void_p(outs[i]), keep=(trees[i], ops[i])) for i in range(n)]


def hm_tune_batched(ops: list, trees: list, fmt: str = "hodlr", opts: list | None = None,
                    candidates=(2, 4, 8, 16), stream=None) -> tuple:
    """Times hm_compress_batched once per candidate concurrency (after one warm-up
    call); returns (best, {candidate: ms})."""
    n = len(ops)
    if len(trees) != n or (opts is not None and len(opts) != n):
        raise ValueError("ops, trees and opts must have the same length")
    opts = opts or [{} for _ in range(n)]
    ops_arr = (_Operator * n)(*[o.op for o in ops])
    trees_arr = (_P * n)(*[t.ptr for t in trees])
    opts_arr = (Opts * n)(*[_opts(**kw) for kw in opts])
    cand = (C.c_int32 * len(candidates))(*candidates)
    ms = (C.c_double * len(candidates))()
    best = C.c_int32()
    fmt_id = {"hodlr": HM_FORMAT_HODLR, "hbsid": HM_FORMAT_HBSID}[fmt]
    _check(lib.hm_tune_batched(n, ops_arr, trees_arr, opts_arr, fmt_id, cand, len(candidates),
                               C.c_void_p(_stream(stream)), C.byref(best), ms), "hm_tune_batched")
    return best.value, {int(c): float(m) for c, m in zip(candidates, ms)}


def hm_apply(h: Handle, trans: int, X: torch.Tensor, Y: torch.Tensor, stream=None) -> None:
    """Y = A_c X (trans 0) or A_c^T X; X, Y given as (ncols, ld) tensors (column-major blocks)."""
    n = h.info["n"]
    px, ldx, ncols = _colmajor(X, n, "X")
    py, ldy, _ = _colmajor(Y, n, "Y")
    _check(lib.hm_apply(h.ptr, trans, ncols, px, ldx, py, ldy, C.c_void_p(_stream(stream))), "hm_apply")


def hm_apply_host(h: Handle, trans: int, X: torch.Tensor, Y: torch.Tensor, stream=None) -> None:
    n = h.info["n"]
    px, ldx, ncols = _colmajor(X, n, "X")
    py, ldy, _ = _colmajor(Y, n, "Y")
    _check(lib.hm_apply_host(h.ptr, trans, ncols, px, ldx, py, ldy, C.c_void_p(_stream(stream))),
           "hm_apply_host")


def hm_reconstruct_block(h: Handle, r0: int, r1: int, c0: int, c1: int, out: torch.Tensor,
                         stream=None) -> None:
    """out: (c1 - c0, ld >= r1 - r0) tensor receiving the column-major block."""
    if out.dim() != 2 or out.stride(1) != 1 or out.shape[0] < c1 - c0 or out.shape[1] < r1 - r0:
        raise ValueError("out must be a (c1 - c0, ld >= r1 - r0) tensor")
    _check(lib.hm_reconstruct_block(h.ptr, r0, r1, c0, c1, _ptr(out), out.stride(0),
                                    C.c_void_p(_stream(stream))), "hm_reconstruct_block")


def hm_rel_frob_error(h: Handle, A: torch.Tensor, stream=None) -> float:
    dtype = {torch.float64: 0, torch.float32: 1}[A.dtype]
    e = C.c_double()
    _check(lib.hm_rel_frob_error(h.ptr, _ptr(A), A.stride(0), dtype, C.byref(e),
                                 C.c_void_p(_stream(stream))), "hm_rel_frob_error")
    return e.value


def hm_info(h: Handle) -> dict:
    i = _Info()
    _check(lib.hm_info(h.ptr, C.byref(i)), "hm_info")
    return {f: getattr(i, f) for f, _ in _Info._fields_}


def hm_node_rank(h: Handle, node: int) -> int:
    k = C.c_int32()
    _check(lib.hm_node_rank(h.ptr, node, C.byref(k)), "hm_node_rank")
    return k.value


HM_FACTOR_APPLY, HM_FACTOR_TRANSPOSE, HM_FACTOR_SOLVE, HM_FACTOR_SOLVE_TRANSPOSE = 0, 1, 2, 3


def hm_product_operator_create(handles: list, kinds: list, alpha: float = 1.0,
                               shift: float = 0.0) -> Operator:
    """Black box alpha F_0 ... F_{nf-1} X + shift X over compressed handles (kinds: HM_FACTOR_*)."""
    nf = len(handles)
    if len(kinds) != nf or nf < 1:
        raise ValueError("one kind per handle, at least one handle")
    arr = (_P * nf)(*[h.ptr for h in handles])
    ks = (C.c_int32 * nf)(*kinds)
    op = _Operator()
    _check(lib.hm_product_operator_create(nf, arr, ks, float(alpha), float(shift), C.byref(op)),
           "hm_product_operator_create")
    return Operator(op, keep=list(handles), product=True)


def hm_save(h: Handle, path: str) -> None:
    """Write the handle's representation to a checkpoint file."""
    _check(lib.hm_save(h.ptr, os.fsencode(path)), "hm_save")


def hm_load(path: str, stream=None) -> Handle:
    """Rebuild a handle from a checkpoint file on the current device."""
    h = C.c_void_p()
    _check(lib.hm_load(os.fsencode(path), C.c_void_p(_stream(stream)), C.byref(h)), "hm_load")
    return Handle(h)


def hm_hodlr_factorize(h: Handle, stream=None) -> None:
    """Factors of the fast direct solver of a HODLR handle (kept by the handle)."""
    _check(lib.hm_hodlr_factorize(h.ptr, C.c_void_p(_stream(stream))), "hm_hodlr_factorize")


def hm_solve(h: Handle, trans: int, B: torch.Tensor, X: torch.Tensor, stream=None) -> None:
    """X = A_c^{-1} B (trans 0) or A_c^{-T} B; B, X as (ncols, ld) tensors (column-major blocks)."""
    n = h.info["n"]
    pb, ldb, ncols = _colmajor(B, n, "B")
    px, ldx, _ = _colmajor(X, n, "X")
    _check(lib.hm_solve(h.ptr, trans, ncols, pb, ldb, px, ldx, C.c_void_p(_stream(stream))), "hm_solve")


def hm_set_profiling(on: bool) -> None:
    """Record a CUDA event at the start of every phase of later compressions."""
    _check(lib.hm_set_profiling(1 if on else 0), "hm_set_profiling")


def hm_profile(h: Handle) -> list:
    """Phase segments of a profiled compression: dicts of level, side, phase name, ms."""
    n = C.c_int32()
    _check(lib.hm_profile(h.ptr, None, 0, C.byref(n)), "hm_profile")
    buf = (_Phase * max(1, n.value))()
    _check(lib.hm_profile(h.ptr, buf, n.value, C.byref(n)), "hm_profile")
    return [{"level": p.level, "side": p.side, "phase": PHASES[p.phase], "ms": p.ms}
            for p in buf[:n.value]]


def hm_skeleton(h: Handle, node: int, side: int) -> list:
    """Global skeleton indices of an HBS-ID node in pivot order (side 0: rows, 1: columns)."""
    r = h.info["r"]
    buf = (C.c_int64 * r)()
    k = C.c_int32()
    _check(lib.hm_skeleton(h.ptr, node, side, buf, C.byref(k)), "hm_skeleton")
    return [int(buf[i]) for i in range(k.value)]


def hm_hodlr_factored_apply(tree: Tree, k: int, U, V, D, x, y, trans: int = 0, stream=None) -> None:
    _check(lib.hm_hodlr_factored_apply(tree.ptr, k, _ptr(U), _ptr(V), _ptr(D), trans, _ptr(x), _ptr(y),
                                       C.c_void_p(_stream(stream))), "hm_hodlr_factored_apply")


def hm_hodlr_factored_apply_noalloc(tree: Tree, k: int, U, V, D, x, y, trans: int = 0,
                                    stream=None) -> None:
    _check(lib.hm_hodlr_factored_apply_noalloc(tree.ptr, k, _ptr(U), _ptr(V), _ptr(D), trans, _ptr(x),
                                               _ptr(y), C.c_void_p(_stream(stream))),
           "hm_hodlr_factored_apply_noalloc")


def hm_hodlr_factored_adjoint(tree: Tree, k: int, U, V, D, x, r, scale=1.0, gx=None, gU=None,
                              gV=None, gD=None, stream=None) -> None:
    _check(lib.hm_hodlr_factored_adjoint(tree.ptr, k, _ptr(U), _ptr(V), _ptr(D), _ptr(x), _ptr(r),
                                         float(scale), _ptr(gx), _ptr(gU), _ptr(gV), _ptr(gD),
                                         C.c_void_p(_stream(stream))), "hm_hodlr_factored_adjoint")


def hm_hodlr_factored_loss_grad(tree: Tree, k: int, U, V, D, x, b, scale=2.0, y=None, r=None,
                                gx=None, gU=None, gV=None, gD=None, stream=None) -> None:
    """y = H x, r = y - b and the adjoint at r (gradients of ||H x - b||^2 at scale 2)."""
    _check(lib.hm_hodlr_factored_loss_grad(tree.ptr, k, _ptr(U), _ptr(V), _ptr(D), _ptr(x),
                                           _ptr(b), float(scale), _ptr(y), _ptr(r), _ptr(gx),
                                           _ptr(gU), _ptr(gV), _ptr(gD),
                                           C.c_void_p(_stream(stream))),
           "hm_hodlr_factored_loss_grad")


def hm_gen_log_kernel(A: torch.Tensor, stream=None) -> None:
    if A.dtype != torch.float32 or A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a row-major float32 CUDA tensor")
    _check(lib.hm_gen_log_kernel(_ptr(A), A.shape[0], A.stride(0), C.c_void_p(_stream(stream))),
           "hm_gen_log_kernel")


def hm_gaussian_test_matrix(tree: Tree, level: int, r: int, seed: int, prec: int, X: torch.Tensor,
                            stream=None) -> None:
    """X: (2r, ld >= n) tensor (column-major n x 2r block), float64 (HM_FP64) or float32."""
    px, ldx, ncols = _colmajor(X, tree.n, "X")
    if ncols < 2 * r:
        raise ValueError("X needs 2r columns")
    _check(lib.hm_gaussian_test_matrix(tree.ptr, level, r, seed, prec, px, ldx,
                                       C.c_void_p(_stream(stream))), "hm_gaussian_test_matrix")


def hm_hodlr_export_level(h: Handle, level: int, U: torch.Tensor, V: torch.Tensor, stream=None) -> None:
    """U, V: (r, n) tensors receiving the column-major n x r factors of the level."""
    _check(lib.hm_hodlr_export_level(h.ptr, level, _ptr(U), _ptr(V), C.c_void_p(_stream(stream))),
           "hm_hodlr_export_level")
