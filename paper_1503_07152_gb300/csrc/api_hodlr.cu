// HODLR compression (Sec. 3, Fig. "Randomized compression of a HODLR matrix")
// and the operations on a compressed handle (apply, transpose apply, block
// reconstruction, Frobenius error, info).
//
// Level l (parents on l, children on l + 1):
//   X = [Omega_2 | Omega_1]                         (Gaussian, Philox)
//   S(:, 0:r) = A Omega_2, S(:, r:2r) = A Omega_1   (two black-box calls, Y_1, Y_2)
//   S -= A^(l) X                                    (peel, levels 1..l)
//   U_child = orth(S(I_child, sample half))         (TSQR + Jacobi + CholQR)
//   X' = [0 U_beta | U_alpha 0]; S = A^T X' - (A^(l))^T X'
//   [V_alpha, B, \hat U_beta] = svd(S(I_alpha, sample half), k | eps)
//   U_beta <- U_beta \hat U_beta B  (the sibling matrix is absorbed into U)
// then the identity probe gives the leaf blocks D.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "hm_api.h"
#include "hm_hodlr.h"

using namespace hm;

namespace hm {

constexpr double kEpsScale = 0.1;  // eps_abs = 0.1 * tol * nu (tolerance reading)

static std::atomic<int> g_profile{0};
bool profiling_on() { return g_profile.load(std::memory_order_relaxed) != 0; }
void set_profiling(int on) { g_profile.store(on ? 1 : 0, std::memory_order_relaxed); }

template <typename T>
void mark(Ctx<T>& c, int level, int side, int phase) {
  if (!c.profile) return;
  typename Ctx<T>::Mark m{level, side, phase, nullptr};
  if (cudaEventCreate(&m.ev) != cudaSuccess) return;
  cudaEventRecord(m.ev, c.st);
  c.marks.push_back(m);
}

template <typename T>
void marks_finish(Ctx<T>& c, hm_handle* h) {
  for (size_t i = 0; i + 1 < c.marks.size(); ++i) {
    float ms = 0.f;
    if (h && cudaEventElapsedTime(&ms, c.marks[i].ev, c.marks[i + 1].ev) == cudaSuccess) {
      hm_phase_t p;
      p.level = c.marks[i].level;
      p.side = c.marks[i].side;
      p.phase = c.marks[i].phase;
      p.ms = ms;
      h->prof.push_back(p);
    }
  }
  for (auto& m : c.marks) cudaEventDestroy(m.ev);
  c.marks.clear();
}

template <typename T>
hm_status box(Ctx<T>& c, int trans, const T* X, T* Y, int64_t ncols, bool ahead) {
  const cudaStream_t st = ahead ? c.la_st : c.st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  // the library's own black boxes get the scratch slot of their stream
  const int rc = library_operator(c.op)
                     ? library_apply(c.op, ahead ? 1 : 0, trans, ncols, X, c.N, Y, c.N, st)
                     : c.op->apply(c.op->ctx, trans, c.N, ncols, X, c.N, Y, c.N, st);
  cudaEventRecord(e1, st);
  c.box_events.push_back({e0, e1});
  if (rc != 0) {
    set_error("black-box apply returned " + std::to_string(rc));
    return HM_ECALLBACK;
  }
  if (trans) c.cols_At += ncols; else c.cols_A += ncols;
  ++c.launches;
  return check_launch("black-box apply");
}

template <typename T>
hm_status la_begin(Ctx<T>& c, const hm_opts* o, cudaStream_t user_st, bool allowed) {
  c.user_st = user_st;
  c.st = user_st;
  c.la = allowed && (o->lookahead == 1 || (o->lookahead == 0 && library_operator(c.op)));
  if (!c.la) return HM_OK;
  int least = 0, greatest = 0;
  HM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  cudaStream_t main_st = nullptr;
  HM_CUDA_TRY(cudaStreamCreateWithPriority(&main_st, cudaStreamNonBlocking, greatest));
  c.st = main_st;
  HM_CUDA_TRY(cudaStreamCreateWithPriority(&c.la_st, cudaStreamNonBlocking, least));
  HM_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_ready, cudaEventDisableTiming));
  HM_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_free, cudaEventDisableTiming));
  HM_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_probe, cudaEventDisableTiming));
  // both streams start after the work already queued on the caller's stream
  HM_CUDA_TRY(cudaEventRecord(c.ev_free, user_st));
  HM_CUDA_TRY(cudaStreamWaitEvent(c.st, c.ev_free, 0));
  HM_CUDA_TRY(cudaStreamWaitEvent(c.la_st, c.ev_free, 0));
  return HM_OK;
}

template <typename T>
hm_status la_join(Ctx<T>& c) {
  if (!c.la) return HM_OK;
  // every look-ahead product has been waited for on c.st (sample_level,
  // sample_identity); c.st's end is the compression's end
  HM_CUDA_TRY(cudaEventRecord(c.ev_ready, c.la_st));
  HM_CUDA_TRY(cudaStreamWaitEvent(c.st, c.ev_ready, 0));
  HM_CUDA_TRY(cudaEventRecord(c.ev_free, c.st));
  HM_CUDA_TRY(cudaStreamWaitEvent(c.user_st, c.ev_free, 0));
  return HM_OK;
}

template <typename T>
void la_end(Ctx<T>& c) {
  if (!c.la) return;
  if (c.la_st) {
    cudaStreamSynchronize(c.la_st);
    cudaStreamDestroy(c.la_st);
  }
  if (c.st && c.st != c.user_st) {
    cudaStreamSynchronize(c.st);
    cudaStreamDestroy(c.st);
  }
  const cudaEvent_t evs[3] = {c.ev_ready, c.ev_free, c.ev_probe};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  c.la_st = nullptr;
  c.ev_ready = c.ev_free = c.ev_probe = nullptr;
  c.st = c.user_st;
  c.la = false;
  c.la_pending = -1;
  c.la_part = 0;
  c.la_cur = -1;
  c.probe_next = 0;
}

// The identity probe's product in pieces of kProbeCols columns (one column
// tile of the sampling GEMM each), so that the look-ahead stream can place them
// in the coarse levels' idle windows; the in-order path takes the same pieces,
// so both give the same products.
constexpr int64_t kProbeCols = 64;

template <typename T>
static int probe_pieces(const Ctx<T>& c) {
  return (int)((c.tree->nmax + kProbeCols - 1) / kProbeCols);
}

template <typename T>
static hm_status probe_piece(Ctx<T>& c, int j, bool ahead) {
  const int64_t c0 = j * kProbeCols;
  const int64_t w = std::min<int64_t>(kProbeCols, c.tree->nmax - c0);
  return box(c, 0, c.XI + c.N * c0, c.YI + c.N * c0, w, ahead);
}

// Look-ahead stream: the next pieces of the identity probe (count of them,
// all that remain if count < 0) after the work enqueued on c.st so far.
template <typename T>
static hm_status la_probe(Ctx<T>& c, int count) {
  const int np = probe_pieces(c);
  if (c.probe_next >= np || count == 0) return HM_OK;
  HM_CUDA_TRY(cudaEventRecord(c.ev_free, c.st));
  HM_CUDA_TRY(cudaStreamWaitEvent(c.la_st, c.ev_free, 0));
  if (c.probe_next == 0)
    launch_identity_probe<T>(c.XI, c.N, c.N, (int)c.tree->nmax, c.tree->d_start, c.tree->L,
                             c.la_st);
  for (int k = 0; c.probe_next < np && (count < 0 || k < count); ++k)
    HM_TRY(probe_piece(c, c.probe_next++, true));
  if (c.probe_next == np) HM_CUDA_TRY(cudaEventRecord(c.ev_probe, c.la_st));
  return HM_OK;
}

// Look-ahead stream: the pending level's test matrix and first half-operator
// product (part 0), its second half (part 1), or whatever of them is pending
// (part 2), after the work enqueued on c.st so far.
template <typename T>
static hm_status la_halves(Ctx<T>& c, int part) {
  if (c.la_pending < 0) return HM_OK;
  const int64_t N = c.N;
  const int r = c.r;
  const int L = c.tree->L;
  const int lv = c.la_pending;
  if (c.la_part == 0 && (part == 0 || part == 2)) {
    // c.st has enqueued everything before this point, the last use of Xa, Sa included
    HM_CUDA_TRY(cudaEventRecord(c.ev_free, c.st));
    HM_CUDA_TRY(cudaStreamWaitEvent(c.la_st, c.ev_free, 0));
    launch_gauss_fill<T>(c.Xa, N, N, r, lv, c.seed, c.bf16, c.tree->d_start, L, c.la_st);
    HM_TRY(box(c, 0, c.Xa, c.Sa, r, true));  // Y_1 = A Omega_2
    c.la_part = 1;
  }
  if (c.la_part == 1 && (part == 1 || part == 2)) {
    HM_CUDA_TRY(cudaEventRecord(c.ev_free, c.st));  // the release point of this half
    HM_CUDA_TRY(cudaStreamWaitEvent(c.la_st, c.ev_free, 0));
    HM_TRY(box(c, 0, c.Xa + N * r, c.Sa + N * r, r, true));  // Y_2 = A Omega_1
    HM_CUDA_TRY(cudaEventRecord(c.ev_ready, c.la_st));
    c.la_part = 0;
    c.la_pending = -1;
  }
  return HM_OK;
}

template <typename T>
hm_status la_release(Ctx<T>& c, int side) {
  if (!c.la) return HM_OK;
  // a level's two half-operator products go out one per side of the current
  // level (each fits beside one side's merges and SVD)
  HM_TRY(la_halves(c, side));
  // the identity probe: one piece per side from level 1 on (the coarse levels'
  // windows have room beside the half-operator products), what is left at the
  // last level's A side
  if (side == 0 && c.la_cur == c.tree->L - 1) return la_probe(c, -1);
  if (c.la_cur >= 1) return la_probe(c, 1);
  return HM_OK;
}

template <typename T>
hm_status sample_level(Ctx<T>& c, int level) {
  const int64_t N = c.N;
  const int r = c.r;
  const int L = c.tree->L;
  if (!c.la) {
    launch_gauss_fill<T>(c.X, N, N, r, level, c.seed, c.bf16, c.tree->d_start, L, c.st);
    HM_TRY(box(c, 0, c.X, c.S, r));                  // Y_1 = A Omega_2
    HM_TRY(box(c, 0, c.X + N * r, c.S + N * r, r));  // Y_2 = A Omega_1
  } else {
    if (level == 0) c.la_pending = 0;
    HM_TRY(la_halves(c, 2));  // level 0, or release points that were not reached
    HM_CUDA_TRY(cudaStreamWaitEvent(c.st, c.ev_ready, 0));
    std::swap(c.X, c.Xa);
    std::swap(c.S, c.Sa);
    c.la_cur = level;
    c.la_pending = level + 1 < L ? level + 1 : -1;  // released from panel_qr
  }
  nonfinite_check_launch(c.S, N * 2 * r, sizeof(T) == 8, c.flags_dev, c.st);
  return HM_OK;
}

template <typename T>
hm_status sample_identity(Ctx<T>& c) {
  if (c.la) {
    HM_TRY(la_probe(c, -1));
    HM_CUDA_TRY(cudaStreamWaitEvent(c.st, c.ev_probe, 0));
    return HM_OK;
  }
  launch_identity_probe<T>(c.XI, c.N, c.N, (int)c.tree->nmax, c.tree->d_start, c.tree->L, c.st);
  for (int j = 0; j < probe_pieces(c); ++j) HM_TRY(probe_piece(c, j, false));
  return HM_OK;
}

// S(:, 0:ncols) -= A^(level) X (or the transpose), node levels 1..level.
template <typename T>
hm_status hodlr_peel(Ctx<T>& c, const T* U, const T* V, int level, const T* X, T* S,
                     int64_t ncols, int trans, double sign) {
  const int64_t N = c.N;
  const int r = c.r;
  for (int j = 1; j <= level; ++j) {
    const LevelPlan& lp = c.tree->plans[j];
    const T* Uj = U + (int64_t)(j - 1) * N * r;
    const T* Vj = V + (int64_t)(j - 1) * N * r;
    const T* Proj = trans ? Uj : Vj;  // projected on the source rows
    const T* Expd = trans ? Vj : Uj;  // expanded on the target rows
    for (int64_t cb = 0; cb < ncols; cb += 128) {
      const int w = (int)std::min<int64_t>(128, ncols - cb);
      launch_seg_tn<T>(lp.d_tn, lp.n_tn, lp.d_tn_begin, lp.nnodes, lp.node0, Proj, N, 0, 0, r,
                       X + cb * N, N, 0, 0, w, c.partial, c.coef, c.st, c.bf16 && sizeof(T) == 8);
      launch_seg_nn<T>(lp.d_nn, lp.n_nn, lp.node0, Expd, N, 0, 0, r, c.coef, (int64_t)r * w, r,
                       1, S + cb * N, N, 0, 0, w, (T)sign, (T)1, c.st, c.bf16 && sizeof(T) == 8);
      c.launches += 3;
    }
  }
  return check_launch("peel");
}

// The panel width pc must fit the shared-memory QR and SVD kernels.
template <typename T>
static hm_status panel_fits(int pc) {
  const size_t lim = 220 * 1024;
  if (pc > 128 || (size_t)(kTsqrRows + 8) * pc * sizeof(T) > lim ||
      (size_t)pc * (pc + 1) * sizeof(T) > lim ||
      (size_t)pc * pc * sizeof(float) + (size_t)pc * pc * (sizeof(T) == 4 ? 4 : 8) + 16 > lim) {
    set_error("panel too wide for the shared-memory QR in this precision");
    return HM_EUNSUPPORTED;
  }
  return HM_OK;
}

// First half of panel_svd: the R factor of every node's panel (TSQR rounds)
// and its SVD (W, sigma per node).
template <typename T>
hm_status panel_qr(Ctx<T>& c, int lv, const T* P, int pc) {
  HM_TRY(panel_fits<T>(pc));
  const LevelPlan& lp = c.tree->plans[lv];
  const int64_t N = c.N;
  mark(c, lv - 1, c.side, HM_PHASE_TSQR);
  for (size_t rd = 0; rd < lp.d_rounds.size(); ++rd) {
    if (sizeof(T) == 8 && c.bf16)  // HM_A32: the Householder work in double-float
      launch_tsqr_df(lp.d_rounds[rd], (int)lp.tsqr_rounds[rd].size(), rd > 0 ? 1 : 0,
                     (const double*)P, N, pc, (double*)c.Rw, c.st);
    else
      launch_tsqr<T>(lp.d_rounds[rd], (int)lp.tsqr_rounds[rd].size(), rd > 0 ? 1 : 0, P, N, pc,
                     c.Rw, c.st);
    // the merges and the SVD that follow leave most SMs idle at the coarse
    // levels: a look-ahead product runs beside them
    if (rd == 0) HM_TRY(la_release(c, c.side));
  }
  mark(c, lv - 1, c.side, HM_PHASE_SVD);
  if (sizeof(T) == 8 && c.bf16)  // HM_A32: the FP64 phases in double-float
    launch_jacobi_df(lp.d_final_slot, lp.nnodes, (const double*)c.Rw, pc, (double*)c.W,
                     (double*)c.sig, c.st);
  else
    launch_jacobi<T>(lp.d_final_slot, lp.nnodes, c.Rw, pc, c.W, c.sig, c.st);
  c.launches += (int)lp.d_rounds.size() + 1;
  return HM_OK;
}

// Second half of panel_svd: rank decision and the orthonormal basis Q (N x r)
// per node of level lv from W, sigma and the panel; when want_m, also the
// coefficients M (pc x r per node).
template <typename T>
hm_status panel_post(Ctx<T>& c, int lv, const T* P, int pc, int mode, int kfix, bool set_eps,
                     T* Q, bool want_m, int32_t* rank_lv) {
  const LevelPlan& lp = c.tree->plans[lv];
  const int64_t N = c.N;
  const int r = c.r;
  // Directions of the sample range below floor_rel * sigma_1 are dropped.  In
  // FP64 the floor sits well above rounding noise (1e-12): directions near the
  // noise level are arbitrary functions of the rounding and would capture an
  // arbitrary share of the coarser levels' truncation error through the
  // transpose peel; what they represent lies far below any tolerance.  In FP32
  // the floor is the unit roundoff.  The tolerance threshold (mode 1) is applied
  // on top.
  const double floor_rel = (sizeof(T) == 4 ? 5.960464477539063e-08
                                           : (mode == 1 ? 1.1102230246251565e-16 : 1e-12));
  launch_truncate<T>(lp.nnodes, c.W, c.sig, pc, r, mode, kfix, kEpsScale * c.tol, c.eps_dev,
                     set_eps ? 1 : 0, floor_rel, rank_lv, c.T1, c.flags_dev + 1, c.st);
  mark(c, lv - 1, c.side, HM_PHASE_ORTH);
  launch_seg_nn<T>(lp.d_nn, lp.n_nn, lp.node0, P, N, 0, 0, pc, c.T1, (int64_t)pc * r, pc, 0, Q,
                   N, 0, 0, r, (T)1, (T)0, c.st, c.bf16 && sizeof(T) == 8);
  launch_seg_tn<T>(lp.d_tn, lp.n_tn, lp.d_tn_begin, lp.nnodes, lp.node0, Q, N, 0, 0, r, Q, N, 0,
                   0, r, c.partial, c.G, c.st, c.bf16 && sizeof(T) == 8);
  launch_cholqr<T>(lp.nnodes, c.G, r, rank_lv, c.T2, c.W, c.sig, pc, c.M, want_m ? 1 : 0, c.st);
  launch_seg_nn<T>(lp.d_nn, lp.n_nn, lp.node0, Q, N, 0, 0, r, c.T2, (int64_t)r * r, r, 0, Q, N, 0,
                   0, r, (T)1, (T)0, c.st, c.bf16 && sizeof(T) == 8);
  c.launches += 7;
  return check_launch("panel svd");
}

// Orthonormal basis / truncated SVD of the panel P (N x pc) per node of level lv.
// Writes Q (N x r) and, when want_m, the coefficients M (pc x r per node).
template <typename T>
hm_status panel_svd(Ctx<T>& c, int lv, const T* P, int pc, int mode, int kfix, bool set_eps,
                    T* Q, bool want_m, int32_t* rank_lv) {
  HM_TRY(panel_qr(c, lv, P, pc));
  return panel_post(c, lv, P, pc, mode, kfix, set_eps, Q, want_m, rank_lv);
}

template <typename T>
hm_status ctx_alloc(Ctx<T>& c, int pc_max, int64_t extra_cols) {
  const int64_t N = c.N;
  const int r = c.r;
  const hm_tree* t = c.tree;
  int max_slots = 0, max_tn = 0;
  for (int lv = 1; lv <= t->L; ++lv) {
    max_slots = std::max(max_slots, t->plans[lv].nslots);
    max_tn = std::max(max_tn, t->plans[lv].n_tn);
  }
  const int64_t nn = (int64_t)1 << t->L;  // most nodes on a level
  auto layout = [&](Arena& a) {
    c.X = a.take<T>(N * 2 * r);
    c.S = a.take<T>(N * 2 * r);
    c.P = a.take<T>(N * pc_max);
    c.Rw = a.take<T>((size_t)max_slots * pc_max * pc_max);
    c.W = a.take<T>(nn * pc_max * pc_max);
    c.sig = a.take<T>(nn * pc_max);
    c.T1 = a.take<T>(nn * pc_max * r);
    c.G = a.take<T>(nn * r * r);
    c.T2 = a.take<T>(nn * r * r);
    c.M = a.take<T>(nn * pc_max * r);
    c.coef = a.take<T>(nn * r * 128);
    c.partial = a.take<double>((size_t)max_tn * 128 * 128);
    c.flags_dev = a.take<int32_t>(4);
    c.eps_dev = a.take<double>(2);
    c.XI = a.take<T>(N * extra_cols);
    c.YI = a.take<T>(N * extra_cols);
    if (c.la) {
      c.Xa = a.take<T>(N * 2 * r);
      c.Sa = a.take<T>(N * 2 * r);
    }
  };
  HM_TRY(arena_alloc(&c.block, layout));
  HM_CUDA_TRY(cudaMemsetAsync(c.flags_dev, 0, 4 * sizeof(int32_t), c.st));
  HM_CUDA_TRY(cudaMemsetAsync(c.eps_dev, 0, 2 * sizeof(double), c.st));
  return HM_OK;
}

template <typename T>
void ctx_free(Ctx<T>& c) {
  for (auto& e : c.box_events) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  c.box_events.clear();
  if (c.block) cudaFree(c.block);
  c.block = nullptr;
}

template <typename T>
double box_ms(Ctx<T>& c) {
  double ms = 0.0;
  for (auto& e : c.box_events) {
    float f = 0.f;
    if (cudaEventElapsedTime(&f, e.first, e.second) == cudaSuccess) ms += f;
  }
  return ms;
}

// One level of the HODLR compression in three stages, around the two panel
// factorizations (panel_qr) of the level:
//   stage A: X = [Omega_2 | Omega_1], S = A X, peel, gather the A-side panel;
//   (panel_qr of the A-side panel)
//   stage B: U bases of the children, X' = [0 U_beta | U_alpha 0], S = A^T X',
//            peel, gather the A^T-side panel;
//   (panel_qr of the A^T-side panel)
//   stage C: V bases, sibling matrices absorbed into U_beta.
template <typename T>
hm_status hodlr_stage_a(Ctx<T>& c, hm_handle* h, int level) {
  const int64_t N = c.N;
  const int r = c.r;
  const int L = c.tree->L;
  const int lv = level + 1;
  T* U = (T*)h->U;
  T* V = (T*)h->V;
  mark(c, level, 0, HM_PHASE_SAMPLE);
  HM_TRY(sample_level(c, level));  // X = [Omega_2 | Omega_1], S = A X
  mark(c, level, 0, HM_PHASE_PEEL);
  HM_TRY(hodlr_peel(c, U, V, level, c.X, c.S, 2 * r, 0, -1.0));
  mark(c, level, 0, HM_PHASE_BASES);
  launch_gather_sample<T>(c.S, N, c.P, N, N, r, lv, c.tree->d_start, L, c.st);
  c.side = 0;
  return HM_OK;
}

template <typename T>
hm_status hodlr_stage_b(Ctx<T>& c, hm_handle* h, int level) {
  const int64_t N = c.N;
  const int r = c.r;
  const int L = c.tree->L;
  const int lv = level + 1;
  T* U = (T*)h->U;
  T* V = (T*)h->V;
  T* Ulv = U + (int64_t)(lv - 1) * N * r;
  HM_TRY(panel_post(c, lv, c.P, r, 0, 0, false, Ulv, false, c.rank_tmp));
  mark(c, level, 1, HM_PHASE_SAMPLE);
  launch_scatter_probe<T>(Ulv, N, c.X, N, N, r, lv, c.tree->d_start, L, c.st);
  HM_TRY(box(c, 1, c.X, c.S, r));                      // Z_1 = A^T Omega_2
  HM_TRY(box(c, 1, c.X + N * r, c.S + N * r, r));      // Z_2 = A^T Omega_1
  nonfinite_check_launch(c.S, N * 2 * r, sizeof(T) == 8, c.flags_dev, c.st);
  mark(c, level, 1, HM_PHASE_PEEL);
  HM_TRY(hodlr_peel(c, U, V, level, c.X, c.S, 2 * r, 1, -1.0));
  mark(c, level, 1, HM_PHASE_BASES);
  launch_gather_sample<T>(c.S, N, c.P, N, N, r, lv, c.tree->d_start, L, c.st);
  c.side = 1;
  return HM_OK;
}

template <typename T>
hm_status hodlr_stage_c(Ctx<T>& c, hm_handle* h, int level) {
  const int64_t N = c.N;
  const int r = c.r;
  const int lv = level + 1;
  T* Ulv = (T*)h->U + (int64_t)(lv - 1) * N * r;
  T* Vlv = (T*)h->V + (int64_t)(lv - 1) * N * r;
  int32_t* rank_lv = c.rank_dev + ((int64_t)1 << lv);
  const int mode = c.mode_tol ? 1 : 2;
  HM_TRY(panel_post(c, lv, c.P, r, mode, c.kfix, level == 0, Vlv, true, rank_lv));
  // U_beta <- U_beta (W_k S_k R2^T) with the coefficients of the sibling's panel
  mark(c, level, 1, HM_PHASE_BASES);
  const LevelPlan& lp = c.tree->plans[lv];
  launch_seg_nn<T>(lp.d_nn, lp.n_nn, lp.node0, Ulv, N, 0, 0, r, c.M, (int64_t)r * r, r, 1, Ulv,
                   N, 0, 0, r, (T)1, (T)0, c.st, c.bf16 && sizeof(T) == 8);
  c.launches += 6;
  return check_launch("hodlr level");
}

// leaf blocks through the identity probe
template <typename T>
hm_status hodlr_leaves(Ctx<T>& c, hm_handle* h) {
  const int64_t N = c.N;
  const int L = c.tree->L;
  const int nmax = (int)c.tree->nmax;
  mark(c, L, 0, HM_PHASE_SAMPLE);
  HM_TRY(sample_identity(c));
  mark(c, L, 0, HM_PHASE_PEEL);
  HM_TRY(hodlr_peel(c, (T*)h->U, (T*)h->V, L, c.XI, c.YI, nmax, 0, -1.0));
  mark(c, L, 0, HM_PHASE_BASES);
  launch_extract_diag<T>(c.YI, N, (T*)h->D, nmax, c.tree->d_start, c.tree->d_size, L, c.st);
  c.launches += 2;
  return check_launch("hodlr diagonal");
}

template <typename T>
hm_status compress_hodlr_t(Ctx<T>& c, hm_handle* h) {
  for (int level = 0; level < c.tree->L; ++level) {
    HM_TRY(hodlr_stage_a(c, h, level));
    HM_TRY(panel_qr(c, level + 1, c.P, c.r));
    HM_TRY(hodlr_stage_b(c, h, level));
    HM_TRY(panel_qr(c, level + 1, c.P, c.r));
    HM_TRY(hodlr_stage_c(c, h, level));
  }
  return hodlr_leaves(c, h);
}

// --------------------------------------------------------------- apply -----
template <typename T>
hm_status hodlr_apply_t(const hm_handle* h, int trans, int64_t ncols, const T* X, int64_t ldx,
                        T* Y, int64_t ldy, cudaStream_t st) {
  const int64_t N = h->n;
  const int r = h->r;
  const hm_tree* t = &h->tree;
  int max_tn = 0;
  for (int lv = 1; lv <= t->L; ++lv) max_tn = std::max(max_tn, t->plans[lv].n_tn);
  const int64_t nn = (int64_t)1 << t->L;
  // contiguous copies of X / Y blocks so that the kernels see ld = N
  const int64_t cbw = 128;
  double* partial = nullptr;
  T *coef = nullptr, *Xc = nullptr, *Yc = nullptr;
  auto layout = [&](Arena& a) {
    partial = a.take<double>((size_t)max_tn * r * cbw);
    coef = a.take<T>(nn * r * cbw);
    Xc = a.take<T>(N * cbw);
    Yc = a.take<T>(N * cbw);
  };
  Arena m;
  layout(m);
  void* blk = nullptr;
  HM_CUDA_TRY(cudaMallocAsync(&blk, m.off + 256, st));
  Arena a;
  a.base = (unsigned char*)blk;
  a.cap = m.off + 256;
  layout(a);
  const T* U = (const T*)h->U;
  const T* V = (const T*)h->V;
  for (int64_t cb = 0; cb < ncols; cb += cbw) {
    const int w = (int)std::min<int64_t>(cbw, ncols - cb);
    launch_copy_cols<T>(X + cb * ldx, ldx, Xc, N, N, w, st);
    launch_fill<T>(Yc, N * w, (T)0, st);
    launch_blockdiag_apply<T>((const T*)h->D, (int)t->nmax, trans, Xc, N, Yc, N, w, t->d_start,
                              t->d_size, t->L, st);
    for (int j = 1; j <= t->L; ++j) {
      const LevelPlan& lp = t->plans[j];
      const T* Uj = U + (int64_t)(j - 1) * N * r;
      const T* Vj = V + (int64_t)(j - 1) * N * r;
      const T* Proj = trans ? Uj : Vj;
      const T* Expd = trans ? Vj : Uj;
      launch_seg_tn<T>(lp.d_tn, lp.n_tn, lp.d_tn_begin, lp.nnodes, lp.node0, Proj, N, 0, 0, r, Xc,
                       N, 0, 0, w, partial, coef, st);
      launch_seg_nn<T>(lp.d_nn, lp.n_nn, lp.node0, Expd, N, 0, 0, r, coef, (int64_t)r * w, r, 1,
                       Yc, N, 0, 0, w, (T)1, (T)1, st);
    }
    launch_copy_cols<T>(Yc, N, Y + cb * ldy, ldy, N, w, st);
  }
  HM_CUDA_TRY(cudaFreeAsync(blk, st));
  return check_launch("hodlr apply");
}

template hm_status hodlr_apply_t<float>(const hm_handle*, int, int64_t, const float*, int64_t,
                                        float*, int64_t, cudaStream_t);
template hm_status hodlr_apply_t<double>(const hm_handle*, int, int64_t, const double*, int64_t,
                                         double*, int64_t, cudaStream_t);

}  // namespace hm

// ------------------------------------------------------------ C entry ------
static hm_status check_opts(const hm_operator* op, const hm_tree* tree, const hm_opts* o,
                            hm_handle** out) {
  if (!op || !op->apply || !tree || !o || !out) {
    set_error("compress: null operator, tree, opts or out");
    return HM_EINVAL;
  }
  if (op->n != tree->n) {
    set_error("compress: operator size differs from the tree size");
    return HM_EINVAL;
  }
  if (o->prec != HM_FP64 && o->prec != HM_MIXED && o->prec != HM_A32) {
    set_error("compress: prec must be HM_FP64 or HM_MIXED");
    return HM_EINVAL;
  }
  if (o->mode_tol) {
    if (!(o->tol > 0.0 && o->tol < 1.0) || o->r < 1) {
      set_error("compress: tolerance mode needs 0 < tol < 1 and r >= 1");
      return HM_EINVAL;
    }
  } else if (o->k < 1 || o->p < 0) {
    set_error("compress: fixed-rank mode needs k >= 1 and p >= 0");
    return HM_EINVAL;
  }
  if (tree->L < 1) {
    set_error("compress: the tree must have at least one level below the root");
    return HM_EINVAL;
  }
  return HM_OK;
}

int opts_r(const hm_opts* o) { return o->mode_tol ? o->r : o->k + o->p; }

namespace hm {

// Allocations and zeroing of one HODLR compression (handle, tree tables,
// factors, context); t0 recorded on the compression's stream.
template <typename T>
hm_status hodlr_begin(HodlrRun<T>& R, const hm_operator* op, hm_tree* tree, const hm_opts* o,
                      cudaStream_t user_st, bool lookahead_allowed) {
  const int r = opts_r(o);
  if (r > 128 || 2 * r > 256) {
    set_error("compress: r must be at most 128");
    return HM_EUNSUPPORTED;
  }
  R.o = o;
  hm_handle* h = new hm_handle();
  R.h = h;
  h->format = HM_FORMAT_HODLR;
  h->prec = o->prec;
  h->n = tree->n;
  h->L = tree->L;
  h->r = r;
  Ctx<T>& c = R.c;
  c.op = op;
  hm_status s = la_begin(c, o, user_st, lookahead_allowed);
  const cudaStream_t st = c.st;  // the compression's stream from here on
  if (s == HM_OK) s = tree_build(tree->n, tree->leaf, &h->tree);
  if (s == HM_OK) s = tree_plans(&h->tree);
  if (s == HM_OK) s = tree_device(&h->tree, st);
  const int64_t N = tree->n;
  if (s == HM_OK) s = device_alloc(&h->U, sizeof(T) * (size_t)tree->L * N * r);
  if (s == HM_OK) s = device_alloc(&h->V, sizeof(T) * (size_t)tree->L * N * r);
  if (s == HM_OK)
    s = device_alloc(&h->D, sizeof(T) * ((size_t)1 << tree->L) * tree->nmax * tree->nmax);
  c.tree = &h->tree;
  c.N = N;
  c.r = r;
  c.seed = o->seed;
  c.mode_tol = o->mode_tol;
  c.kfix = o->k;
  c.tol = o->tol;
  c.bf16 = (o->prec != HM_FP64);
  if (s == HM_OK)
    s = device_alloc((void**)&R.rank_block, sizeof(int32_t) * 2 * ((size_t)1 << (tree->L + 1)));
  c.rank_dev = R.rank_block;
  c.rank_tmp = R.rank_block + ((size_t)1 << (tree->L + 1));
  if (s == HM_OK) s = ctx_alloc(c, r, tree->nmax);
  cudaEventCreate(&R.t0);
  cudaEventCreate(&R.t1);
  c.profile = profiling_on();
  if (s == HM_OK) {
    cudaMemsetAsync(h->U, 0, sizeof(T) * (size_t)tree->L * N * r, st);
    cudaMemsetAsync(h->V, 0, sizeof(T) * (size_t)tree->L * N * r, st);
    cudaMemsetAsync(R.rank_block, 0, sizeof(int32_t) * 2 * ((size_t)1 << (tree->L + 1)), st);
    cudaEventRecord(R.t0, st);
  }
  return s;
}

// After the last stage: t1, synchronization, status flags, ranks and info;
// frees the context.  On success *out receives the handle, otherwise it is
// destroyed.  s is the status of the stages (HM_OK if they all ran).
template <typename T>
hm_status hodlr_end(HodlrRun<T>& R, hm_status s, hm_handle** out) {
  Ctx<T>& c = R.c;
  hm_handle* h = R.h;
  const hm_opts* o = R.o;
  const hm_tree* tree = h ? &h->tree : nullptr;
  const cudaStream_t st = c.st;
  if (s == HM_OK) {
    mark(c, tree->L, 0, -1);  // end of the last phase
    s = la_join(c);
  }
  if (s == HM_OK) {
    cudaEventRecord(R.t1, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error(std::string("compress: ") + cudaGetErrorString(e));
      s = HM_ECUDA;
    }
  }
  // a sampling GEMM whose bounded wait gave up wrote NaN: report the timeout
  // itself rather than the non-finite samples it caused
  if (s == HM_OK) s = dense_take_timeout(c.op);
  int32_t flags[4] = {0, 0, 0, 0};
  double eps[2] = {0, 0};
  const int64_t N = c.N;
  const int r = c.r;
  if (s == HM_OK) {
    cudaMemcpy(flags, c.flags_dev, sizeof(flags), cudaMemcpyDeviceToHost);
    cudaMemcpy(eps, c.eps_dev, sizeof(eps), cudaMemcpyDeviceToHost);
    h->rank.assign((size_t)1 << (tree->L + 1), 0);
    cudaMemcpy(h->rank.data(), R.rank_block, sizeof(int32_t) * h->rank.size(),
               cudaMemcpyDeviceToHost);
    if (flags[0]) {
      set_error("compress: NaN or Inf in the black-box samples");
      s = HM_ENONFINITE;
    } else if (flags[1] && o->strict_rank) {
      set_error("compress: an adaptive rank reached r (raise r)");
      s = HM_ERANK_SATURATED;
    }
  }
  if (s == HM_OK) {
    hm_info_t& in = h->info;
    std::memset(&in, 0, sizeof(in));
    in.format = HM_FORMAT_HODLR;
    in.prec = o->prec;
    in.n = N;
    in.levels = tree->L;
    in.r = r;
    in.max_rank = 0;
    in.min_rank = r;
    for (int64_t a = 2; a < ((int64_t)1 << (tree->L + 1)); ++a) {
      in.max_rank = std::max(in.max_rank, h->rank[a]);
      in.min_rank = std::min(in.min_rank, h->rank[a]);
    }
    in.saturated = flags[1];
    in.cols_A = c.cols_A;
    in.cols_At = c.cols_At;
    in.bytes = (int64_t)(2 * sizeof(T) * (size_t)tree->L * N * r +
                         sizeof(T) * ((size_t)1 << tree->L) * tree->nmax * tree->nmax);
    in.eps_abs = eps[0];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, R.t0, R.t1);
    in.t_compress_ms = ms;
    in.t_blackbox_ms = box_ms(c);
    in.launches = c.launches;
  }
  if (R.t0) cudaEventDestroy(R.t0);
  if (R.t1) cudaEventDestroy(R.t1);
  R.t0 = R.t1 = nullptr;
  marks_finish(c, s == HM_OK ? h : nullptr);
  la_end(c);
  ctx_free(c);
  if (R.rank_block) cudaFree(R.rank_block);
  R.rank_block = nullptr;
  R.h = nullptr;
  if (s != HM_OK) {
    if (h) hm_destroy(h);
    return s;
  }
  *out = h;
  return HM_OK;
}


}  // namespace hm

template <typename T>
static hm_status compress_hodlr_entry(const hm_operator* op, hm_tree* tree, const hm_opts* o,
                                      cudaStream_t st, hm_handle** out) {
  HodlrRun<T> R;
  hm_status s = hodlr_begin(R, op, tree, o, st);
  if (s == HM_OK) s = compress_hodlr_t<T>(R.c, R.h);
  return hodlr_end(R, s, out);
}

extern "C" hm_status hm_compress_hodlr(const hm_operator* op, const hm_tree* tree,
                                       const hm_opts* opts, void* stream, hm_handle** out) {
  clear_error();
  HM_TRY(check_opts(op, tree, opts, out));
  *out = nullptr;
  hm_tree* t = const_cast<hm_tree*>(tree);
  if (opts->prec != HM_MIXED)
    return compress_hodlr_entry<double>(op, t, opts, (cudaStream_t)stream, out);
  return compress_hodlr_entry<float>(op, t, opts, (cudaStream_t)stream, out);
}

namespace hm {
#define HM_INST(T)                                                                          \
  template hm_status box<T>(Ctx<T>&, int, const T*, T*, int64_t, bool);                     \
  template hm_status la_begin<T>(Ctx<T>&, const hm_opts*, cudaStream_t, bool);              \
  template hm_status la_join<T>(Ctx<T>&);                                                   \
  template void la_end<T>(Ctx<T>&);                                                         \
  template hm_status sample_level<T>(Ctx<T>&, int);                                         \
  template hm_status sample_identity<T>(Ctx<T>&);                                           \
  template hm_status la_release<T>(Ctx<T>&, int);                                           \
  template hm_status panel_svd<T>(Ctx<T>&, int, const T*, int, int, int, bool, T*, bool,    \
                                  int32_t*);                                                \
  template hm_status ctx_alloc<T>(Ctx<T>&, int, int64_t);                                   \
  template void ctx_free<T>(Ctx<T>&);                                                       \
  template double box_ms<T>(Ctx<T>&);                                                       \
  template void mark<T>(Ctx<T>&, int, int, int);                                            \
  template void marks_finish<T>(Ctx<T>&, hm_handle*);                                       \
  template hm_status panel_qr<T>(Ctx<T>&, int, const T*, int);                              \
  template hm_status panel_post<T>(Ctx<T>&, int, const T*, int, int, int, bool, T*, bool,   \
                                   int32_t*);                                               \
  template hm_status hodlr_begin<T>(HodlrRun<T>&, const hm_operator*, hm_tree*,             \
                                    const hm_opts*, cudaStream_t, bool);                    \
  template hm_status hodlr_stage_a<T>(Ctx<T>&, hm_handle*, int);                            \
  template hm_status hodlr_stage_b<T>(Ctx<T>&, hm_handle*, int);                            \
  template hm_status hodlr_stage_c<T>(Ctx<T>&, hm_handle*, int);                            \
  template hm_status hodlr_leaves<T>(Ctx<T>&, hm_handle*);                                  \
  template hm_status hodlr_end<T>(HodlrRun<T>&, hm_status, hm_handle**);
HM_INST(float)
HM_INST(double)
#undef HM_INST
}  // namespace hm
