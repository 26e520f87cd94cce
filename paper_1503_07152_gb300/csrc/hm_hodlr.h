// Compression context shared by the HODLR and HBS drivers.
#pragma once

#include <utility>
#include <vector>

#include "hm_api.h"

namespace hm {

template <typename T>
struct Ctx {
  const hm_operator* op = nullptr;
  hm_tree* tree = nullptr;
  cudaStream_t st = nullptr;
  int64_t N = 0;
  int r = 0;
  uint64_t seed = 0;
  int mode_tol = 0, kfix = 0;
  bool bf16 = false;  // test matrices rounded to BF16 values (HM_MIXED, HM_A32)
  double tol = 0.0;
  void* block = nullptr;
  T *X = nullptr, *S = nullptr, *P = nullptr, *Rw = nullptr, *W = nullptr, *sig = nullptr;
  T *T1 = nullptr, *G = nullptr, *T2 = nullptr, *M = nullptr, *coef = nullptr;
  T *XI = nullptr, *YI = nullptr;
  double* partial = nullptr;
  int32_t* flags_dev = nullptr;  // [0] non-finite, [1] saturated ranks
  double* eps_dev = nullptr;
  int32_t* rank_dev = nullptr;   // per heap id
  int32_t* rank_tmp = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> box_events;
  int64_t cols_A = 0, cols_At = 0;
  int launches = 0;
  // phase profile (hm_set_profiling): one event at the start of every phase
  struct Mark {
    int level, side, phase;
    cudaEvent_t ev;
  };
  bool profile = false;
  int side = 0;  // side of the panel being factored (0: A samples, 1: A^T samples)
  std::vector<Mark> marks;
  // Look-ahead sampling (sample_level): the A-side test matrix of a level is a
  // fresh Gaussian block, so its black-box product does not depend on the
  // levels before it.  With `la` set, st is a high-priority stream of the
  // compression's own that joins the caller's stream at both ends, and la_st a
  // low-priority stream on which the next level's samples A Omega (and, during
  // the last level, the identity probe) are computed into Xa, Sa (XI, YI) while
  // st factors the current level's panels.  The look-ahead test matrix and its
  // first half-operator product are released (la_release) once st has launched
  // the first TSQR round of the current level's A-side panel, the last wide
  // launch before the per-node phases that leave most SMs idle; its second
  // half-operator product once st has launched the first TSQR round of the
  // A^T-side panel.  The identity probe's product goes out in 64-column pieces,
  // one per release point from level 1 on.  ev_ready: the look-ahead samples
  // are written; ev_free: st has reached a release point (and is done with the
  // buffers the look-ahead overwrites); ev_probe: the identity probe's samples
  // are written.  la_pending: the level whose samples are released next (-1:
  // none); la_part: how many of its two halves are out.
  bool la = false;
  cudaStream_t user_st = nullptr, la_st = nullptr;
  cudaEvent_t ev_ready = nullptr, ev_free = nullptr, ev_probe = nullptr;
  T *Xa = nullptr, *Sa = nullptr;
  int la_pending = -1, la_part = 0;
  int la_cur = -1;      // the level whose panels c.st is factoring
  int probe_next = 0;   // the next identity-probe piece to release
};

// Records the start of a phase on the compression's stream (no-op unless
// profiling is on).  Phases are the HM_PHASE_* values of hm.h.
template <typename T>
void mark(Ctx<T>& c, int level, int side, int phase);
// Turns the marks into (level, side, phase, ms) segments on the handle and
// destroys the events; the stream has been synchronized.
template <typename T>
void marks_finish(Ctx<T>& c, hm_handle* h);
bool profiling_on();

// One black-box product Y = op(A) X (ncols columns) on the compression's
// stream, or on the look-ahead stream when `ahead` is set.
template <typename T>
hm_status box(Ctx<T>& c, int trans, const T* X, T* Y, int64_t ncols, bool ahead = false);
// Look-ahead set-up (before ctx_alloc): decides whether the compression samples
// one level ahead (o->lookahead: 0 = for the library's own black boxes, 1 =
// always, -1 = never; `allowed` false turns it off) and, if so, creates the two
// streams and makes them wait for the work queued on `user_st`.  Sets c.st.
template <typename T>
hm_status la_begin(Ctx<T>& c, const hm_opts* o, cudaStream_t user_st, bool allowed);
// Makes the caller's stream wait for everything the compression enqueued
// (call after the last launch on c.st; no-op without look-ahead).
template <typename T>
hm_status la_join(Ctx<T>& c);
// Releases the look-ahead streams and events (after c.st has been synchronized
// or on failure; waits for the look-ahead stream first).
template <typename T>
void la_end(Ctx<T>& c);
// Leaves the level's test matrix in c.X (both halves, N x 2r) and its samples
// A X in c.S on c.st, computed there or taken from the look-ahead stream.
template <typename T>
hm_status sample_level(Ctx<T>& c, int level);
// Leaves the identity probe in c.XI and A XI in c.YI on c.st.
template <typename T>
hm_status sample_identity(Ctx<T>& c);
// Release point of the look-ahead stream, reached when c.st has launched the
// first TSQR round of the current level's `side` panel: the pending level's
// half-operator product of that side and, from level 1 on, the next piece of
// the identity probe (all that is left at the last level's A side) start on
// la_st after the work enqueued on c.st so far (no-op without look-ahead).
template <typename T>
hm_status la_release(Ctx<T>& c, int side);
template <typename T>
hm_status panel_svd(Ctx<T>& c, int lv, const T* P, int pc, int mode, int kfix, bool set_eps,
                    T* Q, bool want_m, int32_t* rank_lv);
template <typename T>
hm_status panel_qr(Ctx<T>& c, int lv, const T* P, int pc);
template <typename T>
hm_status panel_post(Ctx<T>& c, int lv, const T* P, int pc, int mode, int kfix, bool set_eps,
                     T* Q, bool want_m, int32_t* rank_lv);
template <typename T>
hm_status ctx_alloc(Ctx<T>& c, int pc_max, int64_t extra_cols);
template <typename T>
void ctx_free(Ctx<T>& c);
template <typename T>
double box_ms(Ctx<T>& c);
template <typename T>
hm_status hodlr_apply_t(const hm_handle* h, int trans, int64_t ncols, const T* X, int64_t ldx,
                        T* Y, int64_t ldy, cudaStream_t st);

// One HODLR compression in flight: its handle, context and timing events.
template <typename T>
struct HodlrRun {
  hm_handle* h = nullptr;
  Ctx<T> c;
  int32_t* rank_block = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  const hm_opts* o = nullptr;
};
// hm_compress_hodlr in pieces, so that a batch can interleave its operators
// level by level: begin (allocations, on `st`), per level stage A, panel_qr,
// stage B, panel_qr, stage C (levels 0 .. L - 1), then the leaves, then end
// (synchronizes the context's stream, fills the handle's ranks and info; on
// failure destroys the handle).
template <typename T>
hm_status hodlr_begin(HodlrRun<T>& R, const hm_operator* op, hm_tree* tree, const hm_opts* o,
                      cudaStream_t st, bool lookahead_allowed = true);
template <typename T>
hm_status hodlr_stage_a(Ctx<T>& c, hm_handle* h, int level);
template <typename T>
hm_status hodlr_stage_b(Ctx<T>& c, hm_handle* h, int level);
template <typename T>
hm_status hodlr_stage_c(Ctx<T>& c, hm_handle* h, int level);
template <typename T>
hm_status hodlr_leaves(Ctx<T>& c, hm_handle* h);
template <typename T>
hm_status hodlr_end(HodlrRun<T>& R, hm_status s, hm_handle** out);

}  // namespace hm

int opts_r(const hm_opts* o);
