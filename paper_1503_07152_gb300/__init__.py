"""GB300 (sm_103a) randomized compression of rank-structured matrices.

Thin Python binding over the C ABI in ``include/hm.h`` (``libhm.so``, built
in-tree by ``paper_1503_07152_gb300.build``).  Every step of the compression,
apply and adjoint runs in the library's CUDA kernels; this module only
marshals arguments (PyTorch tensors provide device memory and streams).
Importing this package loads ``libhm.so`` and fails loudly if it is missing:
there is no CPU fallback.
"""
from ._lib import (  # noqa: F401
    HM_FP64, HM_MIXED, HM_A32, HM_FORMAT_HODLR, HM_FORMAT_HBS, HM_FORMAT_HBSID, HmError, Opts, Tree,
    Operator, Handle, lib, library_path, hm_tree_create, hm_dense_operator_create,
    hm_dense_apply, hm_compress_hodlr, hm_compress_hbs, hm_compress_batched, hm_tune_batched, hm_apply, hm_apply_host,
    hm_reconstruct_block, hm_rel_frob_error, hm_info, hm_node_rank, hm_hodlr_factored_apply, hm_hodlr_factored_apply_noalloc,
    hm_hodlr_factored_adjoint, hm_hodlr_factored_loss_grad, hm_gen_log_kernel, hm_gaussian_test_matrix, hm_hodlr_export_level, hm_version, hm_launch_count, callback_operator,
    hm_dense_operator_check, hm_set_wait_limit, hm_skeleton, hm_set_profiling, hm_profile,
    hm_log_kernel_operator_create, hm_log_kernel_entries, hm_hodlr_factorize, hm_solve, hm_save, hm_load,
    hm_product_operator_create, HM_FACTOR_APPLY, HM_FACTOR_TRANSPOSE, HM_FACTOR_SOLVE,
    HM_FACTOR_SOLVE_TRANSPOSE,
)
from .autograd import HodlrApply  # noqa: F401
