// Host side shared by the entry points: error state, tree construction and the
// per-level work plans (row chunks, TSQR merge schedules) uploaded once per tree,
// the dense black box, and a small device workspace helper.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

#include "hm_api.h"

namespace hm {

static thread_local std::string g_err;
void set_error(const std::string& msg) {
  if (g_err.empty()) g_err = msg;
}
const char* get_error() { return g_err.c_str(); }
void clear_error() { g_err.clear(); }

static std::atomic<long long> g_wait_limit{1ll << 25};
long long wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

static std::atomic<int64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void raise_smem_limit(const void* func, std::atomic<uint32_t>& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 32) return;
  const uint32_t bit = 1u << dev;
  if (done.load(std::memory_order_acquire) & bit) return;
  int optin = 0;
  cudaFuncAttributes fa;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess ||
      cudaFuncGetAttributes(&fa, func) != cudaSuccess)
    return;  // the error stays set: the launch that follows reports it
  // threads that race here all set the same value
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes) == cudaSuccess)
    done.fetch_or(bit, std::memory_order_release);
}

hm_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

// ------------------------------------------------------------ workspace ----
hm_status Workspace::reserve(size_t bytes, cudaStream_t st) {
  (void)st;
  if (bytes <= cap) return HM_OK;
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(&ptr, bytes);
  if (e != cudaSuccess) {
    set_error(std::string("workspace allocation of ") + std::to_string(bytes) + " bytes: " +
              cudaGetErrorString(e));
    return HM_ENOMEM;
  }
  cap = bytes;
  return HM_OK;
}
Workspace::~Workspace() {
  if (ptr) cudaFree(ptr);
}

hm_status device_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return HM_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " +
              cudaGetErrorString(e));
    return HM_ENOMEM;
  }
  return HM_OK;
}

// ----------------------------------------------------------------- plans ----
static void build_chunks(const hm_tree* t, int lv, int64_t maxrows, std::vector<Chunk>& out,
                         std::vector<int32_t>* begin) {
  const int n0 = 1 << lv, n1 = 1 << (lv + 1);
  if (begin) begin->clear();
  for (int node = n0; node < n1; ++node) {
    if (begin) begin->push_back((int32_t)out.size());
    const int64_t s = t->start[node], e = s + t->size[node];
    for (int64_t r = s; r < e; r += maxrows) {
      Chunk c;
      c.node = node;
      c.pad = 0;
      c.r0 = r;
      c.r1 = std::min(e, r + maxrows);
      out.push_back(c);
    }
  }
  if (begin) begin->push_back((int32_t)out.size());
}

static void build_tsqr(const hm_tree* t, int lv, int64_t brows, LevelPlan& lp) {
  const int n0 = 1 << lv, n1 = 1 << (lv + 1);
  std::vector<std::vector<int32_t>> cur(n1 - n0);
  std::vector<TsqrTask> round0;
  int32_t next_slot = 0;
  for (int node = n0; node < n1; ++node) {
    const int64_t s = t->start[node], e = s + t->size[node];
    for (int64_t r = s; r < e; r += brows) {
      TsqrTask tk;
      std::memset(&tk, 0, sizeof(tk));
      tk.node = node;
      tk.nsrc = 1;
      tk.kind[0] = 0;
      tk.r0[0] = r;
      tk.r1[0] = std::min(e, r + brows);
      tk.out_slot = next_slot++;
      cur[node - n0].push_back(tk.out_slot);
      round0.push_back(tk);
    }
  }
  lp.tsqr_rounds.clear();
  lp.tsqr_rounds.push_back(round0);
  for (;;) {
    std::vector<TsqrTask> rnd;
    bool any = false;
    for (int i = 0; i < n1 - n0; ++i) {
      auto& v = cur[i];
      if (v.size() <= 1) continue;
      any = true;
      std::vector<int32_t> nv;
      for (size_t j = 0; j + 1 < v.size(); j += 2) {
        TsqrTask tk;
        std::memset(&tk, 0, sizeof(tk));
        tk.node = n0 + i;
        tk.nsrc = 2;
        tk.kind[0] = tk.kind[1] = 1;
        tk.slot[0] = v[j];
        tk.slot[1] = v[j + 1];
        tk.out_slot = next_slot++;
        nv.push_back(tk.out_slot);
        rnd.push_back(tk);
      }
      if (v.size() % 2) nv.push_back(v.back());
      v.swap(nv);
    }
    if (!any) break;
    lp.tsqr_rounds.push_back(rnd);
  }
  lp.final_slot.resize(n1 - n0);
  for (int i = 0; i < n1 - n0; ++i) lp.final_slot[i] = cur[i][0];
  lp.nslots = next_slot;
}

}  // namespace hm

using namespace hm;

hm_status tree_build(int64_t n, int32_t leaf, hm_tree* t) {
  t->n = n;
  t->leaf = leaf;
  int L = 0;
  while ((n + ((int64_t)1 << L) - 1) / ((int64_t)1 << L) > leaf) ++L;
  if (L > 24) {
    set_error("tree too deep");
    return HM_EINVAL;
  }
  t->L = L;
  const int64_t nn = (int64_t)1 << (L + 1);
  t->start.assign(nn, 0);
  t->size.assign(nn, 0);
  t->size[1] = n;
  for (int64_t tau = 1; tau < ((int64_t)1 << L); ++tau) {
    const int64_t s = t->size[tau];
    t->start[2 * tau] = t->start[tau];
    t->size[2 * tau] = s / 2;
    t->start[2 * tau + 1] = t->start[tau] + s / 2;
    t->size[2 * tau + 1] = s - s / 2;
  }
  t->nmax = 0;
  for (int64_t x = (int64_t)1 << L; x < nn; ++x) t->nmax = std::max(t->nmax, t->size[x]);
  return HM_OK;
}

void tree_free(hm_tree* t) {
  if (t->fdev) cudaFree(t->fdev);
  t->fdev = nullptr;
  if (t->d_start) cudaFree(t->d_start);
  if (t->d_size) cudaFree(t->d_size);
  for (auto& lp : t->plans) {
    if (lp.dev) cudaFree(lp.dev);
    lp.dev = nullptr;
  }
  t->plans.clear();
  t->d_start = t->d_size = nullptr;
}

static void fact_plan_host(hm_tree* t) {
  t->fchunks.clear();
  const int64_t nn = (int64_t)1 << (t->L + 1);
  t->fbegin.assign(nn + 1, 0);
  for (int64_t node = 2; node < nn; ++node) {
    t->fbegin[node] = (int32_t)t->fchunks.size();
    int lv = 0;
    while (((int64_t)1 << (lv + 1)) <= node) ++lv;
    const int64_t s = t->start[node], e = s + t->size[node];
    for (int64_t r = s; r < e; r += 256) {
      FactChunk c;
      c.level = lv;
      c.node = (int32_t)node;
      c.r0 = r;
      c.r1 = std::min(e, r + 256);
      t->fchunks.push_back(c);
    }
  }
  t->fbegin[nn] = (int32_t)t->fchunks.size();
  t->n_fchunks = (int)t->fchunks.size();
}

hm_status tree_plans(hm_tree* t) {
  if (!t->plans.empty()) return HM_OK;
  if (t->L >= 1) fact_plan_host(t);
  t->plans.resize(t->L + 1);
  for (int lv = 1; lv <= t->L; ++lv) {
    LevelPlan& lp = t->plans[lv];
    lp.nnodes = 1 << lv;
    lp.node0 = 1 << lv;
    build_chunks(t, lv, 256, lp.tn, &lp.tn_begin);
    build_chunks(t, lv, 64, lp.nn, nullptr);
    build_tsqr(t, lv, kTsqrRows, lp);
    lp.n_tn = (int)lp.tn.size();
    lp.n_nn = (int)lp.nn.size();
  }
  return HM_OK;
}

// Uploads the node table and the level plans on first use (needs a device).
// The copies go on `st`, and the call waits for them: a plain cudaMemcpy from
// pageable memory may return before its DMA lands, and it runs on the legacy
// stream, which orders nothing on a non-blocking stream, so a kernel launched
// next on such a stream could read a half-written plan.
hm_status tree_device(hm_tree* t, cudaStream_t st) {
  if (t->d_start) return HM_OK;
  std::vector<std::vector<unsigned char>> staged;  // alive until the copies end
  const int64_t nn = (int64_t)1 << (t->L + 1);
  HM_TRY(tree_plans(t));
  auto align = [](size_t b) { return (b + 255) & ~(size_t)255; };
  int64_t* ds = nullptr;
  int64_t* dz = nullptr;
  HM_TRY(device_alloc((void**)&ds, nn * sizeof(int64_t)));
  HM_TRY(device_alloc((void**)&dz, nn * sizeof(int64_t)));
  HM_CUDA_TRY(cudaMemcpyAsync(ds, t->start.data(), nn * sizeof(int64_t), cudaMemcpyHostToDevice,
                              st));
  HM_CUDA_TRY(cudaMemcpyAsync(dz, t->size.data(), nn * sizeof(int64_t), cudaMemcpyHostToDevice,
                              st));
  t->d_size = dz;
  if (t->L >= 1) {
    const size_t b0 = align(t->fchunks.size() * sizeof(FactChunk));
    const size_t bytes = b0 + t->fbegin.size() * sizeof(int32_t);
    HM_TRY(device_alloc(&t->fdev, bytes));
    HM_CUDA_TRY(cudaMemcpyAsync(t->fdev, t->fchunks.data(),
                                t->fchunks.size() * sizeof(FactChunk), cudaMemcpyHostToDevice,
                                st));
    HM_CUDA_TRY(cudaMemcpyAsync((unsigned char*)t->fdev + b0, t->fbegin.data(),
                                t->fbegin.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    t->d_fchunks = (const FactChunk*)t->fdev;
    t->d_fbegin = (const int32_t*)((unsigned char*)t->fdev + b0);
  }
  for (int lv = 1; lv <= t->L; ++lv) {
    LevelPlan& lp = t->plans[lv];
    size_t bytes = 0;
    const size_t o_tn = bytes; bytes = align(bytes + lp.tn.size() * sizeof(Chunk));
    const size_t o_tnb = bytes; bytes = align(bytes + lp.tn_begin.size() * sizeof(int32_t));
    const size_t o_nn = bytes; bytes = align(bytes + lp.nn.size() * sizeof(Chunk));
    std::vector<size_t> o_rounds;
    for (auto& r : lp.tsqr_rounds) {
      o_rounds.push_back(bytes);
      bytes = align(bytes + r.size() * sizeof(TsqrTask));
    }
    const size_t o_fs = bytes; bytes = align(bytes + lp.final_slot.size() * sizeof(int32_t));
    HM_TRY(device_alloc(&lp.dev, bytes));
    staged.emplace_back(bytes, 0);
    std::vector<unsigned char>& host = staged.back();
    std::memcpy(host.data() + o_tn, lp.tn.data(), lp.tn.size() * sizeof(Chunk));
    std::memcpy(host.data() + o_tnb, lp.tn_begin.data(), lp.tn_begin.size() * sizeof(int32_t));
    std::memcpy(host.data() + o_nn, lp.nn.data(), lp.nn.size() * sizeof(Chunk));
    for (size_t i = 0; i < lp.tsqr_rounds.size(); ++i)
      std::memcpy(host.data() + o_rounds[i], lp.tsqr_rounds[i].data(),
                  lp.tsqr_rounds[i].size() * sizeof(TsqrTask));
    std::memcpy(host.data() + o_fs, lp.final_slot.data(), lp.final_slot.size() * sizeof(int32_t));
    HM_CUDA_TRY(cudaMemcpyAsync(lp.dev, host.data(), bytes, cudaMemcpyHostToDevice, st));
    auto base = (unsigned char*)lp.dev;
    lp.d_tn = (const Chunk*)(base + o_tn);
    lp.d_tn_begin = (const int32_t*)(base + o_tnb);
    lp.d_nn = (const Chunk*)(base + o_nn);
    lp.d_rounds.clear();
    for (size_t i = 0; i < lp.tsqr_rounds.size(); ++i)
      lp.d_rounds.push_back((const TsqrTask*)(base + o_rounds[i]));
    lp.d_final_slot = (const int32_t*)(base + o_fs);
  }
  HM_CUDA_TRY(cudaStreamSynchronize(st));
  int dev = -1;
  HM_CUDA_TRY(cudaGetDevice(&dev));
  t->dev = dev;
  t->d_start = ds;  // set last: marks the upload complete
  return HM_OK;
}

extern "C" {

const char* hm_last_error(void) { return get_error(); }
const char* hm_version(void) { return "hm 0.1 (sm_103a)"; }
int64_t hm_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

hm_status hm_tree_create(int64_t n, int32_t leaf_size, hm_tree** out) {
  clear_error();
  if (!out || n < 1 || leaf_size < 1) {
    set_error("hm_tree_create: need n >= 1, leaf_size >= 1 and a non-null out");
    return HM_EINVAL;
  }
  *out = nullptr;
  hm_tree* t = new hm_tree();
  hm_status s = tree_build(n, leaf_size, t);
  if (s == HM_OK) s = tree_plans(t);
  if (s != HM_OK) {
    tree_free(t);
    delete t;
    return s;
  }
  *out = t;
  return HM_OK;
}

void hm_tree_destroy(hm_tree* t) {
  if (!t) return;
  tree_free(t);
  delete t;
}

int32_t hm_tree_levels(const hm_tree* t) { return t ? t->L : -1; }

hm_status hm_tree_node(const hm_tree* t, int64_t node, int64_t* start, int64_t* size) {
  clear_error();
  if (!t || !start || !size || node < 1 || node >= ((int64_t)1 << (t->L + 1))) {
    set_error("hm_tree_node: bad tree, node or output pointer");
    return HM_EINVAL;
  }
  *start = t->start[node];
  *size = t->size[node];
  return HM_OK;
}

// ---------------------------------------------------------- dense box ------
static int dense_slot_apply(hm_dense_ctx* d, int slot, int trans, int64_t n, int64_t ncols,
                            const void* X, int64_t ldx, void* Y, int64_t ldy, cudaStream_t st) {
  if (!d || n != d->n || ncols < 0 || slot < 0 || slot > 1) return 1;
  uint8_t*& flags = slot ? d->flags1 : d->flags;
  void*& xs = slot ? d->xs1 : d->xs;
  int64_t& xs_bytes = slot ? d->xs1_bytes : d->xs_bytes;
  if (!flags && cudaMalloc((void**)&flags, (size_t)d->flags_bytes) != cudaSuccess) {
    flags = nullptr;
    return 3;
  }
  for (int64_t c0 = 0; c0 < ncols; c0 += 1024) {
    const int64_t w = std::min<int64_t>(1024, ncols - c0);
    if (d->dtype == 5) {  // matrix-free log kernel: symmetric, either product
      const int64_t need = gemm_esg_work_bytes(n, w);
      if (need > xs_bytes) {
        if (xs) cudaFree(xs);
        xs = nullptr;
        xs_bytes = 0;
        if (cudaMalloc(&xs, (size_t)need) != cudaSuccess) return 3;
        xs_bytes = need;
      }
      if (launch_gemm_esg_gen(d->tabS, d->tabP, d->aexp, n, w, (const double*)X + c0 * ldx, ldx,
                              (double*)Y + c0 * ldy, ldy, xs, flags, d->err, st) != 0)
        return 2;
    } else if (d->dtype == 0)
      launch_dense_gemm<double>((const double*)d->A, d->lda, trans, n, w,
                                (const double*)X + c0 * ldx, ldx, (double*)Y + c0 * ldy, ldy,
                                flags, st);
    else if (d->dtype == 4 && n <= 524288 && gemm_tc_supported((const float*)d->A, d->lda, n)) {
      const int64_t need = gemm_esg_work_bytes(n, w);
      if (need > xs_bytes) {
        if (xs) cudaFree(xs);
        xs = nullptr;
        xs_bytes = 0;
        if (cudaMalloc(&xs, (size_t)need) != cudaSuccess) return 3;
        xs_bytes = need;
      }
      if (!d->aexp) {
        if (cudaMalloc(&d->aexp, sizeof(int) * 2 * (size_t)gemm_esg_exp_count(n)) != cudaSuccess)
          return 3;
        launch_esg_scales((const float*)d->A, d->lda, n, d->aexp, st);
      }
      if (launch_gemm_esg((const float*)d->A, d->lda, trans, n, w, (const double*)X + c0 * ldx,
                          ldx, (double*)Y + c0 * ldy, ldy, xs, d->aexp, flags, d->err,
                          st) != 0)
        return 2;
    } else if (d->dtype == 2 || d->dtype == 4)
      launch_dense_gemm_a32((const float*)d->A, d->lda, trans, n, w, (const double*)X + c0 * ldx,
                            ldx, (double*)Y + c0 * ldy, ldy, flags, st);
    else if (d->dtype == 1 && gemm_tc_supported((const float*)d->A, d->lda, n)) {
      const int64_t need = 2 * gemm_tc_xs_elems(n, w);
      if (need > xs_bytes) {
        if (xs) cudaFree(xs);
        xs = nullptr;
        xs_bytes = 0;
        if (cudaMalloc(&xs, (size_t)need) != cudaSuccess) return 3;
        xs_bytes = need;
      }
      if (launch_gemm_tc((const float*)d->A, d->lda, trans, n, w, (const float*)X + c0 * ldx,
                         ldx, (float*)Y + c0 * ldy, ldy, xs, flags, d->err, st) != 0)
        return 2;
    } else  // dtype 3, or a layout TMA cannot address: FP32 on the CUDA-core engine
      launch_dense_gemm<float>((const float*)d->A, d->lda, trans, n, w,
                               (const float*)X + c0 * ldx, ldx, (float*)Y + c0 * ldy, ldy,
                               flags, st);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

static int dense_cb(void* ctx, int trans, int64_t n, int64_t ncols, const void* X, int64_t ldx,
                    void* Y, int64_t ldy, void* stream) {
  return dense_slot_apply((hm_dense_ctx*)ctx, 0, trans, n, ncols, X, ldx, Y, ldy,
                          (cudaStream_t)stream);
}

hm_status hm_dense_operator_create(const void* A, int64_t n, int64_t lda, int32_t dtype,
                                   hm_operator* out) {
  clear_error();
  if (!A || !out || n < 1 || lda < n || dtype < 0 || dtype > 4) {
    set_error("hm_dense_operator_create: need A, out, n >= 1, lda >= n, dtype 0..4");
    return HM_EINVAL;
  }
  hm_dense_ctx* d = new hm_dense_ctx();
  d->A = A;
  d->n = n;
  d->lda = lda;
  d->dtype = dtype;
  d->flags_bytes = dense_flags_bytes(n, 1024, dtype == 0);
  hm_status s = device_alloc((void**)&d->flags, (size_t)d->flags_bytes);
  if (s == HM_OK) s = device_alloc((void**)&d->err, sizeof(int));
  // the legacy-stream memset is waited for: the operator may next be applied on
  // a non-blocking stream, which the legacy stream does not order
  if (s == HM_OK && (cudaMemset(d->err, 0, sizeof(int)) != cudaSuccess ||
                     cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess))
    s = HM_ECUDA;
  if (s != HM_OK) {
    if (d->flags) cudaFree(d->flags);
    delete d;
    return s;
  }
  out->apply = dense_cb;
  out->ctx = d;
  out->n = n;
  return HM_OK;
}

hm_status hm_log_kernel_operator_create(int64_t n, hm_operator* out) {
  clear_error();
  if (!out || n < 2 || n > 524288) {
    set_error("hm_log_kernel_operator_create: need 2 <= n <= 524288 and out");
    return HM_EINVAL;
  }
  // tables of the entries' two terms, S[m] = log|sin(pi m / n)| (m >= 1) and
  // P[s] = log(1 + 3 sin^2(pi s / n)) / 2, as float pairs (hi = the FP64 value
  // rounded to FP32, lo = the FP64 remainder rounded to FP32): high parts of
  // all entries first, then the low parts
  const double pi = 3.14159265358979323846;
  const int64_t np = 2 * n - 1;
  std::vector<float> hs((size_t)(2 * n), 0.f), hp((size_t)(2 * np));
  auto put = [](std::vector<float>& v, int64_t i, int64_t stride, double x) {
    const float hi = (float)x;
    v[i] = hi;
    v[stride + i] = (float)(x - (double)hi);
  };
  for (int64_t m = 1; m < n; ++m)
    put(hs, m, n, std::log(std::fabs(std::sin(pi * (double)m / (double)n))));
  for (int64_t t = 0; t < np; ++t) {
    const double sn = std::sin(pi * (double)t / (double)n);
    put(hp, t, np, 0.5 * std::log1p(3.0 * sn * sn));
  }
  hm_dense_ctx* d = new hm_dense_ctx();
  d->n = n;
  d->lda = n;
  d->dtype = 5;
  d->flags_bytes = dense_flags_bytes(n, 1024, 0);
  hm_status s = device_alloc((void**)&d->flags, (size_t)d->flags_bytes);
  if (s == HM_OK) s = device_alloc((void**)&d->err, sizeof(int));
  if (s == HM_OK) s = device_alloc((void**)&d->tabS, sizeof(float) * hs.size());
  if (s == HM_OK) s = device_alloc((void**)&d->tabP, sizeof(float) * hp.size());
  if (s == HM_OK) s = device_alloc((void**)&d->aexp, sizeof(int) * (size_t)gemm_esg_exp_count(n));
  if (s == HM_OK &&
      (cudaMemcpy(d->tabS, hs.data(), sizeof(float) * hs.size(), cudaMemcpyHostToDevice) !=
           cudaSuccess ||
       cudaMemcpy(d->tabP, hp.data(), sizeof(float) * hp.size(), cudaMemcpyHostToDevice) !=
           cudaSuccess ||
       cudaMemset(d->err, 0, sizeof(int)) != cudaSuccess))
    s = HM_ECUDA;
  if (s == HM_OK) {
    launch_logtab_rowexp(d->tabS, d->tabP, n, d->aexp, cudaStreamLegacy);
    if (cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) s = HM_ECUDA;
  }
  if (s != HM_OK) {
    if (s == HM_ECUDA) set_error("hm_log_kernel_operator_create: table upload failed");
    if (d->flags) cudaFree(d->flags);
    if (d->err) cudaFree(d->err);
    if (d->tabS) cudaFree(d->tabS);
    if (d->tabP) cudaFree(d->tabP);
    if (d->aexp) cudaFree(d->aexp);
    delete d;
    return s;
  }
  out->apply = dense_cb;
  out->ctx = d;
  out->n = n;
  return HM_OK;
}

hm_status hm_log_kernel_entries(const hm_operator* op, int64_t r0, int64_t r1, int64_t c0,
                                int64_t c1, float* out, int64_t ld, void* stream) {
  clear_error();
  if (!op || op->apply != dense_cb || !op->ctx || ((hm_dense_ctx*)op->ctx)->dtype != 5 || !out ||
      r0 < 0 || r1 < r0 || r1 > op->n || c0 < 0 || c1 < c0 || c1 > op->n || ld < c1 - c0) {
    set_error("hm_log_kernel_entries: need a matrix-free log-kernel operator, a range inside "
              "[0, n) and ld >= c1 - c0");
    return HM_EINVAL;
  }
  if (r1 == r0 || c1 == c0) return HM_OK;
  const hm_dense_ctx* d = (const hm_dense_ctx*)op->ctx;
  launch_logtab_block(d->tabS, d->tabP, d->n, r0, r1, c0, c1, out, ld, (cudaStream_t)stream);
  return check_launch("hm_log_kernel_entries");
}

void hm_dense_operator_destroy(hm_operator* op) {
  if (!op || !op->ctx) return;
  hm_dense_ctx* d = (hm_dense_ctx*)op->ctx;
  if (d->tabS) cudaFree(d->tabS);
  if (d->tabP) cudaFree(d->tabP);
  if (d->flags) cudaFree(d->flags);
  if (d->xs) cudaFree(d->xs);
  if (d->flags1) cudaFree(d->flags1);
  if (d->xs1) cudaFree(d->xs1);
  if (d->err) cudaFree(d->err);
  if (d->aexp) cudaFree(d->aexp);
  delete d;
  op->ctx = nullptr;
  op->apply = nullptr;
}

}  // extern "C"

bool hm::library_operator(const hm_operator* op) {
  return op && op->apply == dense_cb && op->ctx;
}

int hm::library_apply(const hm_operator* op, int slot, int trans, int64_t ncols, const void* X,
                      int64_t ldx, void* Y, int64_t ldy, cudaStream_t st) {
  if (!library_operator(op)) return 1;
  return dense_slot_apply((hm_dense_ctx*)op->ctx, slot, trans, op->n, ncols, X, ldx, Y, ldy, st);
}

hm_status hm::dense_take_timeout(const hm_operator* op) {
  if (!op || op->apply != dense_cb || !op->ctx) return HM_OK;
  hm_dense_ctx* d = (hm_dense_ctx*)op->ctx;
  int flag = 0;
  HM_CUDA_TRY(cudaMemcpy(&flag, d->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!flag) return HM_OK;
  HM_CUDA_TRY(cudaMemset(d->err, 0, sizeof(int)));
  HM_CUDA_TRY(cudaDeviceSynchronize());
  set_error("a bounded wait of the tensor-core sampling GEMM gave up; its outputs were "
            "written as NaN (see hm_set_wait_limit)");
  return HM_ETIMEOUT;
}

extern "C" {

hm_status hm_set_wait_limit(int64_t polls) {
  clear_error();
  g_wait_limit.store(polls > 0 ? (long long)polls : (1ll << 25), std::memory_order_relaxed);
  return HM_OK;
}

hm_status hm_dense_operator_check(const hm_operator* op, void* stream) {
  clear_error();
  if (!op || !op->ctx || op->apply != dense_cb) {
    set_error("hm_dense_operator_check: need an operator made by hm_dense_operator_create");
    return HM_EINVAL;
  }
  HM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  return dense_take_timeout(op);
}

hm_status hm_dense_apply(const hm_operator* op, int trans, int64_t ncols, const void* X,
                         int64_t ldx, void* Y, int64_t ldy, void* stream) {
  clear_error();
  if (!op || !op->ctx || op->apply != dense_cb || !X || !Y || ncols < 0 || ldx < op->n ||
      ldy < op->n || (trans != 0 && trans != 1)) {
    set_error("hm_dense_apply: need a dense operator, X, Y, ncols >= 0, ld >= n, trans 0|1");
    return HM_EINVAL;
  }
  if (dense_cb(op->ctx, trans, op->n, ncols, X, ldx, Y, ldy, stream) != 0) {
    return check_launch("hm_dense_apply") == HM_OK ? HM_ECUDA : HM_ECUDA;
  }
  return HM_OK;
}

hm_status hm_gen_log_kernel(float* A, int64_t n, int64_t lda, void* stream) {
  clear_error();
  if (!A || n < 1 || lda < n) {
    set_error("hm_gen_log_kernel: need A, n >= 1, lda >= n");
    return HM_EINVAL;
  }
  launch_gen_log_kernel(A, n, lda, (cudaStream_t)stream);
  return check_launch("hm_gen_log_kernel");
}

}  // extern "C"
