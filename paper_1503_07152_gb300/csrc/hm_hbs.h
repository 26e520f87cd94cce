// Declarations of the HBS / HBS-ID kernels.
#pragma once

#include "hm_internal.h"

namespace hm {

// One small GEMM: C (m x n, ldc) = alpha op(A) op(B) + beta C; op = transpose when ta/tb.
struct GemmItem {
  const void* A;
  const void* B;
  void* C;
  int32_t m, n, k;
  int32_t lda, ldb, ldc;
  int32_t ta, tb;
};

template <typename T>
void launch_gather_parent_scaled(const T* U, int64_t ldu, T* P, int64_t ldp, int64_t n, int r,
                                 int lv, const int64_t* d_start, const T* y, int col0,
                                 cudaStream_t st);
template <typename T>
// max_m, max_n, max_k: the largest m, n and k of the items (the tiled form is used
// when its staging fits, else the plain one; the results are the same).  df: FP64
// items in double-float on the FP32 pipe (HM_A32).
void launch_batched_gemm(const GemmItem* items, int count, T alpha, T beta, cudaStream_t st,
                         int max_m, int max_n, int max_k, bool df = false);
template <typename TS, typename TD>
void launch_node_copy(int nnodes, int node0, const TS* src, int64_t sstride, int sld, TD* dst,
                      int64_t dstride, int dld, int rows, int cols, int flip, cudaStream_t st);
template <typename T>
void launch_id_prep_leaf(const T* U, int64_t ldu, const int64_t* d_start, const int64_t* d_size,
                         int L, const T* y, int r, double* Yt, int ncmax, cudaStream_t st);
template <typename T>
void launch_id_prep_parent(int nnodes, int node0, const double* Utmp, const T* y, int r,
                           double* Yt, cudaStream_t st);
// df: the pivoted QR and the substitution in double-float (HM_A32)
void launch_pivqr_id(int nnodes, const double* Yt, int r, int nc, double eps, int kcap,
                     int32_t* k, int32_t* J, double* T, cudaStream_t st, bool df = false);
template <typename T>
void launch_usamp_leaf(const T* U, int64_t ldu, const int64_t* d_start, int L, const int32_t* J,
                       int r, double* Us, int64_t* skel, cudaStream_t st);
void launch_usamp_parent(int nnodes, int node0, const double* Utmp, const int32_t* J, int r,
                         double* Us, int64_t* skel, cudaStream_t st);

}  // namespace hm
