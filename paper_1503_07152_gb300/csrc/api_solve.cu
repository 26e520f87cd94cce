// Fast direct solver for a compressed HODLR matrix (the purpose of the
// compressed formats, Sec. 1: fast matrix inversion; Sec. 2.8 for the format).
//
// With A^(j) the block-diagonal part of A on the nodes of level j (A^(L) = the
// leaf blocks D, A^(0) = A), a parent tau on level j - 1 with children a, b
// gives  A^(j-1)|tau = diag(A^(j)|a, A^(j)|b) (I + W Z^T),
//   W = diag(W_a, W_b),  W_x = (A^(j)|x)^{-1} U_x,  Z^T = [[0, V_b^T], [V_a^T, 0]],
// so A = D (I + W_L Z_L^T) ... (I + W_1 Z_1^T) and, by Sherman-Morrison-Woodbury,
//   (I + W Z^T)^{-1} = I - W M Z^T,  M = (I + Z^T W)^{-1} = [[I, V_b^T W_b], [V_a^T W_a, I]]^{-1}.
// Factorization (bottom-up): D^{-1}; for j = L .. 1: W_j = D^{-1} U_j passed
// through the factors of levels L .. j + 1, then M for every parent of level j.
// Solve: y = D^{-1} b, then y -= W_j M_j Z_j^T y for j = L .. 1; the transposed
// solve runs the transposed factors in the opposite order.  Cost O(k^2 N log^2 N)
// to factor, O(k N log N) per solve; the same segmented kernels as the
// compression, FP64 (double-float products for HM_A32 handles).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "hm_hbs.h"
#include "hm_hodlr.h"

using namespace hm;

namespace {

template <typename T>
struct SolveCtx {
  const hm_handle* h = nullptr;
  cudaStream_t st = nullptr;
  bool df = false;
  int64_t N = 0;
  int r = 0, L = 0;
  T *Dinv = nullptr, *W = nullptr, *M = nullptr;
  T* q = nullptr;  // per node of a level: r x w projections
  T* s = nullptr;  // per node of a level: r x w coefficients
  double* partial = nullptr;
  GemmItem* items = nullptr;
  size_t items_cap = 0;
  std::vector<GemmItem> v;

  void add(const T* A, int lda, int ta, const T* B, int ldb, T* C, int ldc, int m, int n, int k) {
    GemmItem it;
    it.A = A; it.B = B; it.C = C;
    it.m = m; it.n = n; it.k = k;
    it.lda = lda; it.ldb = ldb; it.ldc = ldc;
    it.ta = ta; it.tb = 0;
    v.push_back(it);
  }
  hm_status run(T beta) {
    if (v.empty()) return HM_OK;
    if (v.size() > items_cap) {
      set_error("internal: too many solver GEMM items");
      return HM_EUNSUPPORTED;
    }
    HM_CUDA_TRY(cudaMemcpyAsync(items, v.data(), v.size() * sizeof(GemmItem),
                                cudaMemcpyHostToDevice, st));
    int mm = 0, nn = 0, kk = 0;
    for (const GemmItem& g : v) {
      mm = std::max(mm, (int)g.m);
      nn = std::max(nn, (int)g.n);
      kk = std::max(kk, (int)g.k);
    }
    launch_batched_gemm<T>(items, (int)v.size(), (T)1, beta, st, mm, nn, kk);
    v.clear();
    return check_launch("solver gemm");
  }

  // Y (N x w, ld N) <- (I + W_j Z_j^T)^{-1} Y  (trans = 0)
  //                 or (I + Z_j W_j^T)^{-1} Y  (trans = 1, the transposed factor)
  hm_status level_inverse(int j, T* Y, int w, int trans) {
    const LevelPlan& lp = h->tree.plans[j];
    const T* Wj = W + (int64_t)(j - 1) * N * r;
    const T* Vj = (const T*)h->V + (int64_t)(j - 1) * N * r;
    const T* Proj = trans ? Wj : Vj;  // q_x = Proj_x^T y_x
    const T* Expd = trans ? Vj : Wj;  // y_x -= Expd_x s_x
    const int64_t rw = (int64_t)r * w, rr2 = (int64_t)4 * r * r;
    launch_seg_tn<T>(lp.d_tn, lp.n_tn, lp.d_tn_begin, lp.nnodes, lp.node0, Proj, N, 0, 0, r, Y, N,
                     0, 0, w, partial, q, st, df);
    // s = M [q_b; q_a] (forward) or M^T [q_a; q_b] (transposed), split per child;
    // then y_a -= W_a s_a, y_b -= W_b s_b (forward) or y_a -= V_a s_a, y_b -= V_b s_b
    // with s_a = (M^T [q_a; q_b])[r:2r], s_b = (...)[0:r] (transposed)
    const int np = lp.nnodes / 2;
    for (int pass = 0; pass < 2; ++pass) {
      for (int pi = 0; pi < np; ++pi) {
        const T* Mp = M + (int64_t)((1 << (j - 1)) - 1 + pi) * rr2;  // parents of levels < j first
        const T* qa = q + (int64_t)(2 * pi) * rw;
        const T* qb = q + (int64_t)(2 * pi + 1) * rw;
        T* sa = s + (int64_t)(2 * pi) * rw;
        T* sb = s + (int64_t)(2 * pi + 1) * rw;
        const int n2 = 2 * r;
        if (!trans) {
          // s_a = M[0:r, 0:r] q_b + M[0:r, r:2r] q_a ; s_b = M[r:2r, 0:r] q_b + M[r:2r, r:2r] q_a
          const T* in = pass == 0 ? qb : qa;
          const int coff = pass == 0 ? 0 : r;
          add(Mp + (int64_t)coff * n2, n2, 0, in, r, sa, r, r, w, r);
          add(Mp + r + (int64_t)coff * n2, n2, 0, in, r, sb, r, r, w, r);
        } else {
          // u = M^T [q_a; q_b]; s_b = u[0:r] (-> V_b), s_a = u[r:2r] (-> V_a)
          // u[0:r] = M[0:r, 0:r]^T q_a + M[r:2r, 0:r]^T q_b
          // u[r:2r] = M[0:r, r:2r]^T q_a + M[r:2r, r:2r]^T q_b
          const T* in = pass == 0 ? qa : qb;
          const int roff = pass == 0 ? 0 : r;
          add(Mp + roff, n2, 1, in, r, sb, r, r, w, r);
          add(Mp + roff + (int64_t)r * n2, n2, 1, in, r, sa, r, r, w, r);
        }
      }
      HM_TRY(run(pass == 0 ? (T)0 : (T)1));
    }
    launch_seg_nn<T>(lp.d_nn, lp.n_nn, lp.node0, Expd, N, 0, 0, r, s, rw, r, 0, Y, N, 0, 0, w,
                     (T)-1, (T)1, st, df);
    return check_launch("solver level");
  }
};

template <typename T>
hm_status factorize_t(hm_handle* h, cudaStream_t st) {
  const hm_tree* t = &h->tree;
  const int64_t N = h->n;
  const int r = h->r, L = h->L, nmax = (int)t->nmax, nleaf = 1 << L;
  if (nmax > 256 || 2 * r > 256) {
    set_error("hm_hodlr_factorize: leaves of at most 256 points and r <= 128 are supported");
    return HM_EUNSUPPORTED;
  }
  const int64_t nparents = ((int64_t)1 << L) - 1;
  // handle storage: Dinv, W (L levels of N x r), M (one 2r x 2r per parent)
  const int64_t e_dinv = (int64_t)nleaf * nmax * nmax, e_w = (int64_t)L * N * r,
                e_m = nparents * 4 * r * r;
  void* blk = nullptr;
  HM_TRY(device_alloc(&blk, sizeof(T) * (size_t)(e_dinv + e_w + e_m)));
  T* Dinv = (T*)blk;
  T* Wall = Dinv + e_dinv;
  T* Mall = Wall + e_w;
  // scratch: Gauss-Jordan work, per-node projections, partials, GEMM items
  int max_tn = 0;
  for (int lv = 1; lv <= L; ++lv) max_tn = std::max(max_tn, t->plans[lv].n_tn);
  const int64_t gj = std::max<int64_t>((int64_t)nleaf * nmax * 2 * nmax,
                                       (nparents + 1) / 2 * 8 * (int64_t)r * r);
  SolveCtx<T> c;
  T* work = nullptr;
  int* sing = nullptr;
  void* scr = nullptr;
  c.items_cap = 4 * (size_t)nleaf + 16;
  auto layout = [&](Arena& a) {
    work = a.take<T>((size_t)gj);
    c.q = a.take<T>((size_t)nleaf * r * r);
    c.s = a.take<T>((size_t)nleaf * r * r);
    c.partial = a.take<double>((size_t)max_tn * r * r);
    c.items = a.take<GemmItem>(c.items_cap);
    sing = a.take<int>(1);
  };
  hm_status s = arena_alloc(&scr, layout);
  if (s != HM_OK) {
    cudaFree(blk);
    return s;
  }
  c.h = h; c.st = st; c.df = (h->prec == HM_A32); c.N = N; c.r = r; c.L = L;
  c.Dinv = Dinv; c.W = Wall; c.M = Mall;
  cudaMemsetAsync(sing, 0, sizeof(int), st);
  // leaf inverses
  launch_gj_load_leaves<T>((const T*)h->D, nmax, t->d_size, L, work, st);
  launch_gauss_jordan<T>(work, nleaf, nmax, Dinv, sing, st);
  for (int j = L; j >= 1 && s == HM_OK; --j) {
    T* Wj = Wall + (int64_t)(j - 1) * N * r;
    const T* Uj = (const T*)h->U + (int64_t)(j - 1) * N * r;
    // W_j = D^{-1} U_j, then through the factors of the finer levels
    launch_fill<T>(Wj, N * r, (T)0, st);
    launch_blockdiag_apply<T>(Dinv, nmax, 0, Uj, N, Wj, N, r, t->d_start, t->d_size, L, st);
    for (int i = L; i > j && s == HM_OK; --i) s = c.level_inverse(i, Wj, r, 0);
    if (s != HM_OK) break;
    // M for the parents of level j: P_x = V_x^T W_x per child x on level j
    const LevelPlan& lp = t->plans[j];
    const T* Vj = (const T*)h->V + (int64_t)(j - 1) * N * r;
    launch_seg_tn<T>(lp.d_tn, lp.n_tn, lp.d_tn_begin, lp.nnodes, lp.node0, Vj, N, 0, 0, r, Wj, N,
                     0, 0, r, c.partial, c.q, st, c.df);
    const int np = lp.nnodes / 2;
    launch_gj_load_woodbury<T>(c.q, r, np, work, st);
    launch_gauss_jordan<T>(work, np, 2 * r, Mall + (int64_t)((1 << (j - 1)) - 1) * 4 * r * r,
                           sing, st);
    s = check_launch("hm_hodlr_factorize");
  }
  int hs = 0;
  if (s == HM_OK) {
    cudaError_t e = cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error(std::string("hm_hodlr_factorize: ") + cudaGetErrorString(e));
      s = HM_ECUDA;
    } else if (hs) {
      set_error("hm_hodlr_factorize: a leaf block or a Woodbury matrix is singular");
      s = HM_ENONFINITE;
    }
  } else {
    cudaStreamSynchronize(st);
  }
  cudaFree(scr);
  if (s != HM_OK) {
    cudaFree(blk);
    return s;
  }
  if (h->solv) cudaFree(h->solv);
  h->solv = blk;
  h->solv_dinv = 0;
  h->solv_w = e_dinv;
  h->solv_m = e_dinv + e_w;
  return HM_OK;
}

template <typename T>
hm_status solve_t(const hm_handle* h, int trans, int64_t ncols, const T* B, int64_t ldb, T* X,
                  int64_t ldx, cudaStream_t st) {
  const hm_tree* t = &h->tree;
  const int64_t N = h->n;
  const int r = h->r, L = h->L, nmax = (int)t->nmax, nleaf = 1 << L;
  const int64_t cbw = 128;
  int max_tn = 0;
  for (int lv = 1; lv <= L; ++lv) max_tn = std::max(max_tn, t->plans[lv].n_tn);
  SolveCtx<T> c;
  c.h = h; c.st = st; c.df = (h->prec == HM_A32); c.N = N; c.r = r; c.L = L;
  c.Dinv = (T*)h->solv + h->solv_dinv;
  c.W = (T*)h->solv + h->solv_w;
  c.M = (T*)h->solv + h->solv_m;
  c.items_cap = 4 * (size_t)nleaf + 16;
  T *Yc = nullptr, *Bc = nullptr;
  auto layout = [&](Arena& a) {
    Yc = a.take<T>((size_t)N * cbw);
    Bc = a.take<T>((size_t)N * cbw);
    c.q = a.take<T>((size_t)nleaf * r * cbw);
    c.s = a.take<T>((size_t)nleaf * r * cbw);
    c.partial = a.take<double>((size_t)max_tn * r * cbw);
    c.items = a.take<GemmItem>(c.items_cap);
  };
  Arena m;
  layout(m);
  void* blk = nullptr;
  HM_CUDA_TRY(cudaMallocAsync(&blk, m.off + 256, st));
  Arena a;
  a.base = (unsigned char*)blk;
  a.cap = m.off + 256;
  layout(a);
  hm_status s = HM_OK;
  for (int64_t cb = 0; cb < ncols && s == HM_OK; cb += cbw) {
    const int w = (int)std::min<int64_t>(cbw, ncols - cb);
    launch_copy_cols<T>(B + cb * ldb, ldb, Bc, N, N, w, st);
    if (!trans) {
      launch_fill<T>(Yc, N * w, (T)0, st);
      launch_blockdiag_apply<T>(c.Dinv, nmax, 0, Bc, N, Yc, N, w, t->d_start, t->d_size, L, st);
      for (int j = L; j >= 1 && s == HM_OK; --j) s = c.level_inverse(j, Yc, w, 0);
    } else {
      for (int j = 1; j <= L && s == HM_OK; ++j) s = c.level_inverse(j, Bc, w, 1);
      launch_fill<T>(Yc, N * w, (T)0, st);
      launch_blockdiag_apply<T>(c.Dinv, nmax, 1, Bc, N, Yc, N, w, t->d_start, t->d_size, L, st);
    }
    if (s == HM_OK) launch_copy_cols<T>(Yc, N, X + cb * ldx, ldx, N, w, st);
  }
  cudaFreeAsync(blk, st);
  if (s != HM_OK) return s;
  return check_launch("hm_solve");
}

}  // namespace

extern "C" hm_status hm_hodlr_factorize(hm_handle* h, void* stream) {
  clear_error();
  if (!h || h->format != HM_FORMAT_HODLR) {
    set_error("hm_hodlr_factorize: need a HODLR handle");
    return HM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (h->prec == HM_MIXED) return factorize_t<float>(h, st);
  return factorize_t<double>(h, st);
}

extern "C" hm_status hm_solve(const hm_handle* h, int trans, int64_t ncols, const void* B,
                              int64_t ldb, void* X, int64_t ldx, void* stream) {
  clear_error();
  if (!h || h->format != HM_FORMAT_HODLR || !h->solv || !B || !X || ncols < 0 || ldb < h->n ||
      ldx < h->n || (trans != 0 && trans != 1)) {
    set_error("hm_solve: need a factorized HODLR handle (hm_hodlr_factorize), B, X, "
              "ncols >= 0, ld >= n, trans 0|1");
    return HM_EINVAL;
  }
  if (ncols == 0) return HM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->prec == HM_MIXED)
    return solve_t<float>(h, trans, ncols, (const float*)B, ldb, (float*)X, ldx, st);
  return solve_t<double>(h, trans, ncols, (const double*)B, ldb, (double*)X, ldx, st);
}

// ------------------------------------------------------ operator products ---
// Black boxes built from compressed handles (Sec. 5.2: a product such as
// S (I/2 + D)^{-1} is compressed by peeling it through its factors' fast
// applies and solves).
namespace {

struct ProductCtx {
  std::vector<const hm_handle*> hs;
  std::vector<int32_t> kinds;
  double alpha = 1.0, shift = 0.0;
  int64_t n = 0;
  int32_t prec = 0;
};

// one factor: dst = op(h) src
hm_status apply_factor(const hm_handle* h, int kind, int64_t ncols, const void* src, int64_t lds,
                       void* dst, int64_t ldd, void* stream) {
  switch (kind) {
    case HM_FACTOR_APPLY: return hm_apply(h, 0, ncols, src, lds, dst, ldd, stream);
    case HM_FACTOR_TRANSPOSE: return hm_apply(h, 1, ncols, src, lds, dst, ldd, stream);
    case HM_FACTOR_SOLVE: return hm_solve(h, 0, ncols, src, lds, dst, ldd, stream);
    default: return hm_solve(h, 1, ncols, src, lds, dst, ldd, stream);
  }
}

template <typename T>
int product_cb_t(ProductCtx* p, int trans, int64_t n, int64_t ncols, const T* X, int64_t ldx, T* Y,
                 int64_t ldy, cudaStream_t st) {
  const int nf = (int)p->hs.size();
  T* tmp[2] = {nullptr, nullptr};
  const size_t bytes = sizeof(T) * (size_t)n * (size_t)ncols;
  if (cudaMallocAsync((void**)&tmp[0], bytes, st) != cudaSuccess) return 3;
  if (cudaMallocAsync((void**)&tmp[1], bytes, st) != cudaSuccess) {
    cudaFreeAsync(tmp[0], st);
    return 3;
  }
  const T* cur = X;
  int64_t ldc = ldx;
  int rc = 0;
  for (int s = 0; s < nf && rc == 0; ++s) {
    // op = F_0 ... F_{nf-1}: the rightmost factor first; the transpose runs the
    // transposed factors in the opposite order
    const int i = trans ? s : nf - 1 - s;
    int kind = p->kinds[i];
    if (trans) kind ^= 1;  // apply <-> transpose, solve <-> transposed solve
    T* dst = tmp[s & 1];
    if (apply_factor(p->hs[i], kind, ncols, cur, ldc, dst, n, st) != HM_OK) rc = 5;
    cur = dst;
    ldc = n;
  }
  if (rc == 0)
    launch_axpby<T>(Y, ldy, (T)p->alpha, cur, ldc, (T)p->shift, X, ldx, n, ncols, st);
  cudaFreeAsync(tmp[0], st);
  cudaFreeAsync(tmp[1], st);
  if (rc == 0 && cudaGetLastError() != cudaSuccess) rc = 2;
  return rc;
}

int product_cb(void* ctx, int trans, int64_t n, int64_t ncols, const void* X, int64_t ldx,
               void* Y, int64_t ldy, void* stream) {
  ProductCtx* p = (ProductCtx*)ctx;
  if (!p || n != p->n || ncols < 0) return 1;
  if (ncols == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (p->prec == HM_MIXED)
    return product_cb_t<float>(p, trans, n, ncols, (const float*)X, ldx, (float*)Y, ldy, st);
  return product_cb_t<double>(p, trans, n, ncols, (const double*)X, ldx, (double*)Y, ldy, st);
}

}  // namespace

extern "C" hm_status hm_product_operator_create(int32_t nf, const hm_handle* const* handles,
                                                const int32_t* kinds, double alpha, double shift,
                                                hm_operator* out) {
  clear_error();
  if (nf < 1 || !handles || !kinds || !out) {
    set_error("hm_product_operator_create: need nf >= 1 handles and kinds, and out");
    return HM_EINVAL;
  }
  const int64_t n = handles[0] ? handles[0]->n : 0;
  const bool single = handles[0] && handles[0]->prec == HM_MIXED;
  for (int32_t i = 0; i < nf; ++i) {
    const hm_handle* h = handles[i];
    if (!h || h->n != n || (h->prec == HM_MIXED) != single || kinds[i] < 0 || kinds[i] > 3) {
      set_error("hm_product_operator_create: factor " + std::to_string(i) +
                ": null handle, another n, another element type or a bad kind");
      return HM_EINVAL;
    }
    if (kinds[i] >= HM_FACTOR_SOLVE && (h->format != HM_FORMAT_HODLR || !h->solv)) {
      set_error("hm_product_operator_create: factor " + std::to_string(i) +
                " is a solve: it needs a HODLR handle factorized by hm_hodlr_factorize");
      return HM_EINVAL;
    }
  }
  ProductCtx* p = new ProductCtx();
  p->hs.assign(handles, handles + nf);
  p->kinds.assign(kinds, kinds + nf);
  p->alpha = alpha;
  p->shift = shift;
  p->n = n;
  p->prec = handles[0]->prec;
  out->apply = product_cb;
  out->ctx = p;
  out->n = n;
  return HM_OK;
}

extern "C" void hm_product_operator_destroy(hm_operator* op) {
  if (!op || op->apply != product_cb || !op->ctx) return;
  delete (ProductCtx*)op->ctx;
  op->ctx = nullptr;
  op->apply = nullptr;
}
