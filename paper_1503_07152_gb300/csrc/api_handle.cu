// Operations on a compressed handle: apply / transpose apply (device and host
// buffers), dense block reconstruction, the relative Frobenius error against a
// dense operator (Sec. 5), info, ranks, destruction; and the factored HODLR
// apply with its hand-written adjoint.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "hm_hodlr.h"

using namespace hm;

namespace hm {
void set_profiling(int on);
template <typename T>
hm_status hbs_apply_t(const hm_handle* h, int trans, int64_t ncols, const T* X, int64_t ldx,
                      T* Y, int64_t ldy, cudaStream_t st);
void hbs_free(hm_handle* h);
}  // namespace hm

template <typename T>
static hm_status apply_any(const hm_handle* h, int trans, int64_t ncols, const T* X, int64_t ldx,
                           T* Y, int64_t ldy, cudaStream_t st) {
  if (h->format == HM_FORMAT_HODLR) return hodlr_apply_t<T>(h, trans, ncols, X, ldx, Y, ldy, st);
  return hbs_apply_t<T>(h, trans, ncols, X, ldx, Y, ldy, st);
}

static size_t elem(const hm_handle* h) { return h->prec == HM_MIXED ? 4 : 8; }

extern "C" {

hm_status hm_apply(const hm_handle* h, int trans, int64_t ncols, const void* X, int64_t ldx,
                   void* Y, int64_t ldy, void* stream) {
  clear_error();
  if (!h || !X || !Y || ncols < 0 || ldx < h->n || ldy < h->n || (trans != 0 && trans != 1)) {
    set_error("hm_apply: need handle, X, Y, ncols >= 0, ld >= n, trans 0|1");
    return HM_EINVAL;
  }
  if (ncols == 0) return HM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->prec != HM_MIXED)
    return apply_any<double>(h, trans, ncols, (const double*)X, ldx, (double*)Y, ldy, st);
  return apply_any<float>(h, trans, ncols, (const float*)X, ldx, (float*)Y, ldy, st);
}

hm_status hm_apply_host(const hm_handle* h, int trans, int64_t ncols, const void* X_host,
                        int64_t ldx, void* Y_host, int64_t ldy, void* stream) {
  clear_error();
  if (!h || !X_host || !Y_host || ncols < 0 || ldx < h->n || ldy < h->n) {
    set_error("hm_apply_host: need handle, X, Y, ncols >= 0, ld >= n");
    return HM_EINVAL;
  }
  if (ncols == 0) return HM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = elem(h);
  const int64_t N = h->n;
  void* dx = nullptr;
  void* dy = nullptr;
  HM_CUDA_TRY(cudaMallocAsync(&dx, es * N * ncols, st));
  HM_CUDA_TRY(cudaMallocAsync(&dy, es * N * ncols, st));
  HM_CUDA_TRY(cudaMemcpy2DAsync(dx, es * N, X_host, es * ldx, es * N, ncols,
                                cudaMemcpyHostToDevice, st));
  hm_status s = hm_apply(h, trans, ncols, dx, N, dy, N, stream);
  if (s == HM_OK) {
    cudaError_t e = cudaMemcpy2DAsync(Y_host, es * ldy, dy, es * N, es * N, ncols,
                                      cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
      set_error(std::string("hm_apply_host copy back: ") + cudaGetErrorString(e));
      s = HM_ECUDA;
    }
  }
  cudaFreeAsync(dx, st);
  cudaFreeAsync(dy, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (s == HM_OK && e != cudaSuccess) {
    set_error(std::string("hm_apply_host: ") + cudaGetErrorString(e));
    s = HM_ECUDA;
  }
  return s;
}

}  // extern "C"

template <typename T>
static hm_status reconstruct_t(const hm_handle* h, int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                               T* out, int64_t ld, cudaStream_t st) {
  const int64_t N = h->n;
  const int64_t cw = 256;
  T* X = nullptr;
  T* Y = nullptr;
  HM_CUDA_TRY(cudaMallocAsync((void**)&X, sizeof(T) * N * cw, st));
  HM_CUDA_TRY(cudaMallocAsync((void**)&Y, sizeof(T) * N * cw, st));
  hm_status s = HM_OK;
  for (int64_t c = c0; c < c1 && s == HM_OK; c += cw) {
    const int64_t w = std::min(cw, c1 - c);
    launch_identity_cols<T>(X, N, N, c, w, st);
    s = apply_any<T>(h, 0, w, X, N, Y, N, st);
    if (s == HM_OK) launch_copy_cols<T>(Y + r0, N, out + (c - c0) * ld, ld, r1 - r0, w, st);
  }
  cudaFreeAsync(X, st);
  cudaFreeAsync(Y, st);
  if (s != HM_OK) return s;
  return check_launch("hm_reconstruct_block");
}

template <typename T, typename TA = T>
static hm_status frob_t(const hm_handle* h, const TA* A, int64_t lda, double* err, cudaStream_t st) {
  const int64_t N = h->n;
  const int64_t cw = 256;
  T* X = nullptr;
  T* Y = nullptr;
  double* acc = nullptr;
  HM_CUDA_TRY(cudaMallocAsync((void**)&X, sizeof(T) * N * cw, st));
  HM_CUDA_TRY(cudaMallocAsync((void**)&Y, sizeof(T) * N * cw, st));
  HM_CUDA_TRY(cudaMallocAsync((void**)&acc, 2 * sizeof(double), st));
  HM_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
  hm_status s = HM_OK;
  for (int64_t c = 0; c < N && s == HM_OK; c += cw) {
    const int64_t w = std::min(cw, N - c);
    launch_identity_cols<T>(X, N, N, c, w, st);
    s = apply_any<T>(h, 0, w, X, N, Y, N, st);
    if (s == HM_OK) {
      if constexpr (std::is_same<T, TA>::value) launch_frob_tile<T>(A, lda, Y, N, N, c, w, acc, st);
      else launch_frob_tile_a32((const float*)A, lda, (const double*)Y, N, N, c, w, acc, st);
    }
  }
  double hacc[2] = {0, 0};
  if (s == HM_OK) {
    cudaError_t e = cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error(std::string("hm_rel_frob_error: ") + cudaGetErrorString(e));
      s = HM_ECUDA;
    }
  }
  cudaFreeAsync(X, st);
  cudaFreeAsync(Y, st);
  cudaFreeAsync(acc, st);
  if (s == HM_OK) *err = hacc[1] > 0 ? std::sqrt(hacc[0] / hacc[1]) : 0.0;
  return s;
}

extern "C" {

hm_status hm_reconstruct_block(const hm_handle* h, int64_t r0, int64_t r1, int64_t c0,
                               int64_t c1, void* out, int64_t ld, void* stream) {
  clear_error();
  if (!h || !out || r0 < 0 || r1 < r0 || r1 > h->n || c0 < 0 || c1 < c0 || c1 > h->n ||
      ld < std::max<int64_t>(1, r1 - r0)) {
    set_error("hm_reconstruct_block: bad range, ld or null pointer");
    return HM_EINVAL;
  }
  if (r1 == r0 || c1 == c0) return HM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->prec != HM_MIXED) return reconstruct_t<double>(h, r0, r1, c0, c1, (double*)out, ld, st);
  return reconstruct_t<float>(h, r0, r1, c0, c1, (float*)out, ld, st);
}

hm_status hm_rel_frob_error(const hm_handle* h, const void* A, int64_t lda, int32_t dtype,
                            double* err, void* stream) {
  clear_error();
  if (!h || !A || !err || lda < h->n || dtype != (h->prec == HM_FP64 ? 0 : 1)) {
    set_error("hm_rel_frob_error: need handle, A (double for HM_FP64, float otherwise), lda >= n");
    return HM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (h->prec == HM_FP64) return frob_t<double>(h, (const double*)A, lda, err, st);
  if (h->prec == HM_A32) return frob_t<double, float>(h, (const float*)A, lda, err, st);
  return frob_t<float>(h, (const float*)A, lda, err, st);
}

hm_status hm_info(const hm_handle* h, hm_info_t* out) {
  clear_error();
  if (!h || !out) {
    set_error("hm_info: null handle or out");
    return HM_EINVAL;
  }
  *out = h->info;
  return HM_OK;
}

hm_status hm_node_rank(const hm_handle* h, int64_t node, int32_t* rank) {
  clear_error();
  if (!h || !rank || node < 2 || node >= ((int64_t)1 << (h->L + 1))) {
    set_error("hm_node_rank: bad handle, node or rank pointer");
    return HM_EINVAL;
  }
  if (h->format == HM_FORMAT_HODLR) *rank = h->rank[node ^ 1];
  else if (h->format == HM_FORMAT_HBSID) *rank = h->kin[node];
  else *rank = h->r;
  return HM_OK;
}

hm_status hm_set_profiling(int32_t on) {
  clear_error();
  set_profiling(on);
  return HM_OK;
}

hm_status hm_profile(const hm_handle* h, hm_phase_t* out, int32_t cap, int32_t* count) {
  clear_error();
  if (!h || !count || cap < 0 || (cap > 0 && !out)) {
    set_error("hm_profile: need handle, count, cap >= 0 and out when cap > 0");
    return HM_EINVAL;
  }
  const int32_t n = (int32_t)h->prof.size();
  for (int32_t i = 0; i < n && i < cap; ++i) out[i] = h->prof[i];
  *count = n;
  return HM_OK;
}

hm_status hm_skeleton(const hm_handle* h, int64_t node, int32_t side, int64_t* idx, int32_t* k) {
  clear_error();
  if (!h || h->format != HM_FORMAT_HBSID || !h->skel || !idx || !k || node < 2 ||
      node >= ((int64_t)1 << (h->L + 1)) || (side != 0 && side != 1)) {
    set_error("hm_skeleton: need an HBS-ID handle, 2 <= node < 2^(L+1), side 0|1, idx, k");
    return HM_EINVAL;
  }
  const int64_t nheap = (int64_t)1 << (h->L + 1);
  const int32_t kk = side == 0 ? h->kin[node] : h->kout[node];
  const int64_t* src = h->skel + (int64_t)side * nheap * h->r + node * h->r;
  HM_CUDA_TRY(cudaMemcpy(idx, src, sizeof(int64_t) * (size_t)h->r, cudaMemcpyDeviceToHost));
  for (int32_t a = kk; a < h->r; ++a) idx[a] = -1;
  *k = kk;
  return HM_OK;
}

void hm_destroy(hm_handle* h) {
  if (!h) return;
  if (h->solv) cudaFree(h->solv);
  if (h->U) cudaFree(h->U);
  if (h->V) cudaFree(h->V);
  if (h->D) cudaFree(h->D);
  hbs_free(h);
  tree_free(&h->tree);
  delete h;
}

// ------------------------------------------------ factored HODLR + adjoint --
hm_status hm_hodlr_factored_apply(const hm_tree* tree, int32_t k, const float* U, const float* V,
                                  const float* D, int trans, const float* x, float* y,
                                  void* stream) {
  clear_error();
  if (!tree || k < 1 || k > 64 || !U || !V || !D || !x || !y || tree->L < 1 ||
      (trans != 0 && trans != 1)) {
    set_error("hm_hodlr_factored_apply: need tree (L >= 1), 1 <= k <= 64, U, V, D, x, y");
    return HM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  HM_TRY(factored_check(tree, false));
  HM_TRY(tree_device(const_cast<hm_tree*>(tree), st));
  float* scratch = nullptr;
  const size_t sbytes = factored_scratch_bytes(tree, k);
  HM_CUDA_TRY(cudaMallocAsync((void**)&scratch, sbytes, st));
  launch_factored_apply(tree, k, U, V, D, trans, x, y, scratch, st);
  cudaFreeAsync(scratch, st);
  return check_launch("hm_hodlr_factored_apply");
}

hm_status hm_hodlr_factored_adjoint(const hm_tree* tree, int32_t k, const float* U,
                                    const float* V, const float* D, const float* x,
                                    const float* res, float scale, float* gx, float* gU, float* gV,
                                    float* gD, void* stream) {
  clear_error();
  if (!tree || k < 1 || k > 64 || !U || !V || !D || !x || !res || tree->L < 1) {
    set_error("hm_hodlr_factored_adjoint: need tree (L >= 1), 1 <= k <= 64, U, V, D, x, res");
    return HM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  HM_TRY(factored_check(tree, true));
  HM_TRY(tree_device(const_cast<hm_tree*>(tree), st));
  float* scratch = nullptr;
  const size_t sbytes = factored_scratch_bytes(tree, k);
  HM_CUDA_TRY(cudaMallocAsync((void**)&scratch, sbytes, st));
  launch_factored_adjoint(tree, k, U, V, D, x, res, scale, gx, gU, gV, gD, scratch, st);
  cudaFreeAsync(scratch, st);
  return check_launch("hm_hodlr_factored_adjoint");
}

hm_status hm_hodlr_factored_loss_grad(const hm_tree* tree, int32_t k, const float* U,
                                      const float* V, const float* D, const float* x,
                                      const float* b, float scale, float* y, float* res,
                                      float* gx, float* gU, float* gV, float* gD, void* stream) {
  clear_error();
  if (!tree || k < 1 || k > 64 || !U || !V || !D || !x || !b || tree->L < 1) {
    set_error("hm_hodlr_factored_loss_grad: need tree (L >= 1), 1 <= k <= 64, U, V, D, x, b");
    return HM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  HM_TRY(factored_check(tree, false));
  HM_TRY(factored_check(tree, true));
  HM_TRY(tree_device(const_cast<hm_tree*>(tree), st));
  float* scratch = nullptr;
  const size_t sbytes = factored_loss_grad_scratch_bytes(tree, k);
  HM_CUDA_TRY(cudaMallocAsync((void**)&scratch, sbytes, st));
  launch_factored_loss_grad(tree, k, U, V, D, x, b, scale, y, res, gx, gU, gV, gD, scratch, st);
  cudaFreeAsync(scratch, st);
  return check_launch("hm_hodlr_factored_loss_grad");
}

}  // extern "C"

extern "C" hm_status hm_gaussian_test_matrix(const hm_tree* tree, int32_t level, int32_t r,
                                            uint64_t seed, int32_t prec, void* X, int64_t ldx,
                                            void* stream) {
  clear_error();
  if (!tree || !X || level < 0 || level >= tree->L || r < 1 || ldx < tree->n ||
      (prec != HM_FP64 && prec != HM_MIXED && prec != HM_A32)) {
    set_error("hm_gaussian_test_matrix: need tree, X, 0 <= level < L, r >= 1, ldx >= n, prec");
    return HM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  HM_TRY(tree_device(const_cast<hm_tree*>(tree), st));
  if (prec != HM_MIXED)
    launch_gauss_fill<double>((double*)X, ldx, tree->n, r, level, seed, prec == HM_A32,
                              tree->d_start, tree->L, st);
  else
    launch_gauss_fill<float>((float*)X, ldx, tree->n, r, level, seed, true, tree->d_start, tree->L,
                             st);
  return check_launch("hm_gaussian_test_matrix");
}

extern "C" hm_status hm_hodlr_export_level(const hm_handle* h, int32_t level, void* U, void* V,
                                          void* stream) {
  clear_error();
  if (!h || h->format != HM_FORMAT_HODLR || level < 1 || level > h->L || !U || !V) {
    set_error("hm_hodlr_export_level: need a HODLR handle, 1 <= level <= L, U and V");
    return HM_EINVAL;
  }
  const size_t es = h->prec == HM_MIXED ? 4 : 8;
  const size_t bytes = es * (size_t)h->n * h->r;
  const size_t off = bytes * (size_t)(level - 1);
  cudaStream_t st = (cudaStream_t)stream;
  HM_CUDA_TRY(cudaMemcpyAsync(U, (const char*)h->U + off, bytes, cudaMemcpyDeviceToDevice, st));
  HM_CUDA_TRY(cudaMemcpyAsync(V, (const char*)h->V + off, bytes, cudaMemcpyDeviceToDevice, st));
  return HM_OK;
}
