// Batched compression of independent operators: many operators of uneven size
// and rank compressed in one call.
//
// HODLR (the batch workload: many small operators, whose per-node panel
// factorizations are latency-bound) runs level-synchronously from one host
// thread: for every level the operators' black-box products, peels and gathers
// are issued on a few streams, and then ONE launch per TSQR round and ONE
// launch of the panel SVD cover the nodes of that level of every operator
// (NodeJob lists, in HM_A32 where those kernels are the double-float ones); the
// per-operator streams wait on it through events.  Each node's arithmetic is
// that of the one-operator call, so every handle equals the one-call result.
// HBS-ID runs the one-operator path concurrently from a pool of host threads.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <memory>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "hm_api.h"
#include "hm_hodlr.h"

using namespace hm;

namespace {

// The level-wide job lists of a batch: for every level lv and TSQR round rd the
// tasks of every operator that has that round, then the SVD of every node.
struct ForestPlan {
  std::vector<NodeJob> host;
  // per level (index lv): per round (offset, count, cmax), and the SVD (offset, count, cmax)
  struct Span {
    int64_t off = 0;
    int count = 0, cmax = 0;
  };
  std::vector<std::vector<Span>> rounds;
  std::vector<Span> svd;
  NodeJob* dev = nullptr;
};

hm_status forest_build(ForestPlan& F, std::vector<std::unique_ptr<HodlrRun<double>>>& runs,
                       const std::vector<int>& members, int maxL) {
  F.rounds.assign(maxL + 1, {});
  F.svd.assign(maxL + 1, {});
  for (int lv = 1; lv <= maxL; ++lv) {
    size_t nr = 0;
    for (int i : members)
      if (runs[i]->h->tree.L >= lv) nr = std::max(nr, runs[i]->h->tree.plans[lv].d_rounds.size());
    F.rounds[lv].resize(nr);
    for (size_t rd = 0; rd < nr; ++rd) {
      ForestPlan::Span sp;
      sp.off = (int64_t)F.host.size();
      for (int i : members) {
        Ctx<double>& c = runs[i]->c;
        const hm_tree& t = runs[i]->h->tree;
        if (t.L < lv || rd >= t.plans[lv].d_rounds.size()) continue;
        const LevelPlan& lp = t.plans[lv];
        for (size_t k = 0; k < lp.tsqr_rounds[rd].size(); ++k) {
          NodeJob j{};
          j.task = lp.d_rounds[rd] + k;
          j.P = c.P;
          j.ldp = c.N;
          j.R = c.Rw;
          j.c = c.r;
          F.host.push_back(j);
        }
        sp.cmax = std::max(sp.cmax, c.r);
      }
      sp.count = (int)((int64_t)F.host.size() - sp.off);
      F.rounds[lv][rd] = sp;
    }
    ForestPlan::Span sv;
    sv.off = (int64_t)F.host.size();
    for (int i : members) {
      Ctx<double>& c = runs[i]->c;
      const hm_tree& t = runs[i]->h->tree;
      if (t.L < lv) continue;
      const LevelPlan& lp = t.plans[lv];
      const int64_t cc = (int64_t)c.r * c.r;
      for (int k = 0; k < lp.nnodes; ++k) {
        NodeJob j{};
        j.R = c.Rw + (int64_t)lp.final_slot[k] * cc;
        j.W = c.W + (int64_t)k * cc;
        j.sigma = c.sig + (int64_t)k * c.r;
        j.c = c.r;
        F.host.push_back(j);
      }
      sv.cmax = std::max(sv.cmax, c.r);
    }
    sv.count = (int)((int64_t)F.host.size() - sv.off);
    F.svd[lv] = sv;
  }
  if (F.host.empty()) return HM_OK;
  HM_CUDA_TRY(cudaMalloc((void**)&F.dev, sizeof(NodeJob) * F.host.size()));
  HM_CUDA_TRY(cudaMemcpy(F.dev, F.host.data(), sizeof(NodeJob) * F.host.size(),
                         cudaMemcpyHostToDevice));
  return HM_OK;
}

// Level-synchronous HODLR compression of the operators `members` (all of element
// type T).  streams: the per-operator streams (operator i on streams[i % S]);
// main: the stream of the level-wide launches.  On failure *failed names the
// operator and every handle of the group is destroyed.
template <typename T>
hm_status batched_hodlr(const std::vector<int>& members, const hm_operator* ops,
                        hm_tree* const* trees, const hm_opts* opts,
                        const std::vector<cudaStream_t>& streams, cudaStream_t main,
                        hm_handle** outs, int32_t* failed) {
  const int S = (int)streams.size();
  std::vector<std::unique_ptr<HodlrRun<T>>> runs(members.empty() ? 0 : members.back() + 1);
  std::vector<int> started;
  hm_status s = HM_OK;
  int bad = -1;
  for (int i : members) {
    runs[i].reset(new HodlrRun<T>());
    s = hodlr_begin(*runs[i], &ops[i], trees[i], &opts[i], streams[i % S], false);
    started.push_back(i);
    if (s != HM_OK) { bad = i; break; }
  }
  int maxL = 0;
  if (s == HM_OK)
    for (int i : members) maxL = std::max(maxL, (int)runs[i]->h->tree.L);
  // the level-wide panel factorizations (HM_A32 operators: double-float kernels
  // over job lists); operators of the other precisions factor their panels on
  // their own streams
  std::vector<int> forest, single;
  for (int i : members) {
    const bool df = sizeof(T) == 8 && opts[i].prec == HM_A32;
    (df ? forest : single).push_back(i);
  }
  ForestPlan F;
  if constexpr (std::is_same<T, double>::value)
    if (s == HM_OK && !forest.empty()) s = forest_build(F, runs, forest, maxL);
  std::vector<cudaEvent_t> ev(S, nullptr);
  cudaEvent_t ev_main = nullptr;
  for (int k = 0; k < S && s == HM_OK; ++k)
    if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess) s = HM_ECUDA;
  if (s == HM_OK && cudaEventCreateWithFlags(&ev_main, cudaEventDisableTiming) != cudaSuccess)
    s = HM_ECUDA;
  // every forest operator's stream -> main, the level-wide launches, main -> every stream
  auto panel_qr_all = [&](int level, const std::vector<int>& act) -> hm_status {
    const int lv = level + 1;
    bool any = false;
    for (int i : act) {
      const bool df = sizeof(T) == 8 && opts[i].prec == HM_A32;
      if (!df) {
        HM_TRY(panel_qr(runs[i]->c, lv, runs[i]->c.P, runs[i]->c.r));
        continue;
      }
      any = true;
    }
    if (!any) return HM_OK;
    for (int k = 0; k < S; ++k) {
      HM_CUDA_TRY(cudaEventRecord(ev[k], streams[k]));
      HM_CUDA_TRY(cudaStreamWaitEvent(main, ev[k], 0));
    }
    const auto& rounds = F.rounds[lv];
    for (size_t rd = 0; rd < rounds.size(); ++rd)
      launch_tsqr_df_jobs(F.dev + rounds[rd].off, rounds[rd].count, rd > 0 ? 1 : 0,
                          rounds[rd].cmax, main);
    launch_jacobi_df_jobs(F.dev + F.svd[lv].off, F.svd[lv].count, F.svd[lv].cmax, main);
    HM_TRY(check_launch("batched panel factorization"));
    HM_CUDA_TRY(cudaEventRecord(ev_main, main));
    for (int k = 0; k < S; ++k) HM_CUDA_TRY(cudaStreamWaitEvent(streams[k], ev_main, 0));
    for (int i : act)
      if (sizeof(T) == 8 && opts[i].prec == HM_A32)
        runs[i]->c.launches += (int)rounds.size() + 1;
    return HM_OK;
  };
  // operators whose tree has fewer levels than the deepest drop out early
  for (int level = 0; level < maxL && s == HM_OK; ++level) {
    std::vector<int> act;
    for (int i : members)
      if ((int)runs[i]->h->tree.L > level) act.push_back(i);
    for (int i : act)
      if (s == HM_OK && (s = hodlr_stage_a(runs[i]->c, runs[i]->h, level)) != HM_OK) bad = i;
    if (s == HM_OK && (s = panel_qr_all(level, act)) != HM_OK) bad = act.front();
    for (int i : act)
      if (s == HM_OK && (s = hodlr_stage_b(runs[i]->c, runs[i]->h, level)) != HM_OK) bad = i;
    if (s == HM_OK && (s = panel_qr_all(level, act)) != HM_OK) bad = act.front();
    for (int i : act) {
      if (s == HM_OK && (s = hodlr_stage_c(runs[i]->c, runs[i]->h, level)) != HM_OK) bad = i;
      if (s == HM_OK && (int)runs[i]->h->tree.L == level + 1 &&
          (s = hodlr_leaves(runs[i]->c, runs[i]->h)) != HM_OK)
        bad = i;
    }
  }
  if (s == HM_OK && cudaStreamSynchronize(main) != cudaSuccess) {
    set_error("hm_compress_batched: the level-wide launches failed");
    s = HM_ECUDA;
  }
  const std::string msg = s == HM_OK ? std::string() : std::string(hm_last_error());
  // every started compression ends (synchronizes its stream, frees its context)
  for (int i : started) {
    hm_handle* out = nullptr;
    const hm_status e = hodlr_end(*runs[i], s == HM_OK ? HM_OK : HM_ECUDA, &out);
    outs[i] = out;
    if (s == HM_OK && e != HM_OK) {
      s = e;
      bad = i;
    }
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (ev_main) cudaEventDestroy(ev_main);
  if (F.dev) cudaFree(F.dev);
  if (s != HM_OK) {
    for (int i : members) {
      if (outs[i]) hm_destroy(outs[i]);
      outs[i] = nullptr;
    }
    if (!msg.empty()) {
      clear_error();
      set_error(msg);
    }
    *failed = bad < 0 ? 0 : bad;
  }
  return s;
}

}  // namespace

extern "C" hm_status hm_compress_batched(int32_t nops, const hm_operator* ops,
                                         hm_tree* const* trees, const hm_opts* opts,
                                         int32_t format, int32_t max_concurrency, void* stream,
                                         hm_handle** outs) {
  clear_error();
  if (nops < 0 || (nops > 0 && (!ops || !trees || !opts || !outs)) ||
      (format != HM_FORMAT_HODLR && format != HM_FORMAT_HBSID) || max_concurrency < 0) {
    set_error("hm_compress_batched: need nops >= 0, ops, trees, opts, outs, format HODLR or "
              "HBSID, max_concurrency >= 0");
    return HM_EINVAL;
  }
  for (int32_t i = 0; i < nops; ++i) outs[i] = nullptr;
  if (nops == 0) return HM_OK;
  for (int32_t i = 0; i < nops; ++i)
    if (!trees[i]) {
      set_error("hm_compress_batched: trees[" + std::to_string(i) + "] is null");
      return HM_EINVAL;
    }
  int dev = 0;
  HM_CUDA_TRY(cudaGetDevice(&dev));
  // upload every tree's tables here, once, so that the workers never race on a
  // tree shared between operators
  for (int32_t i = 0; i < nops; ++i) HM_TRY(tree_device(trees[i], (cudaStream_t)stream));
  // the workers' streams start after the work already queued on `stream`
  cudaEvent_t ready;
  HM_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  HM_CUDA_TRY(cudaEventRecord(ready, (cudaStream_t)stream));
  if (format == HM_FORMAT_HODLR) {
    // level-synchronous, one host thread; the operators of each element type
    // form one group
    const int S = std::min<int>(nops, max_concurrency > 0 ? max_concurrency : 8);
    std::vector<cudaStream_t> streams(S, nullptr);
    hm_status s = HM_OK;
    for (int k = 0; k < S && s == HM_OK; ++k) {
      if (cudaStreamCreateWithFlags(&streams[k], cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamWaitEvent(streams[k], ready, 0) != cudaSuccess) {
        set_error("hm_compress_batched: could not create a stream");
        s = HM_ECUDA;
      }
    }
    std::vector<int> g64, g32;
    for (int32_t i = 0; i < nops; ++i) (opts[i].prec == HM_MIXED ? g32 : g64).push_back(i);
    int32_t failed = 0;
    if (s == HM_OK && !g64.empty())
      s = batched_hodlr<double>(g64, ops, trees, opts, streams, (cudaStream_t)stream, outs,
                                &failed);
    if (s == HM_OK && !g32.empty())
      s = batched_hodlr<float>(g32, ops, trees, opts, streams, (cudaStream_t)stream, outs,
                               &failed);
    for (auto st : streams)
      if (st) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
      }
    cudaEventDestroy(ready);
    if (s != HM_OK) {
      for (int32_t j = 0; j < nops; ++j) {
        if (outs[j]) hm_destroy(outs[j]);
        outs[j] = nullptr;
      }
      const std::string m = hm_last_error();
      clear_error();  // the first error is kept: restate it with the operator's index
      set_error("hm_compress_batched: operator " + std::to_string(failed) + ": " + m);
    }
    return s;
  }
  const int nthr = std::min<int>(nops, max_concurrency > 0 ? max_concurrency : 8);
  std::atomic<int32_t> next{0};
  std::vector<hm_status> status(nops, HM_OK);
  std::vector<std::string> msg(nops);
  auto worker = [&]() {
    cudaSetDevice(dev);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
    if (s) cudaStreamWaitEvent(s, ready, 0);
    for (;;) {
      const int32_t i = next.fetch_add(1);
      if (i >= nops) break;
      if (!s) {
        status[i] = HM_ECUDA;
        msg[i] = "could not create a stream";
        continue;
      }
      const hm_status r =
          format == HM_FORMAT_HODLR ? hm_compress_hodlr(&ops[i], trees[i], &opts[i], s, &outs[i])
                                    : hm_compress_hbs(&ops[i], trees[i], &opts[i], s, &outs[i]);
      status[i] = r;
      if (r != HM_OK) msg[i] = hm_last_error();
    }
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nthr; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  cudaEventDestroy(ready);
  for (int32_t i = 0; i < nops; ++i)
    if (status[i] != HM_OK) {
      for (int32_t j = 0; j < nops; ++j) {
        if (outs[j]) hm_destroy(outs[j]);
        outs[j] = nullptr;
      }
      set_error("hm_compress_batched: operator " + std::to_string(i) + ": " + msg[i]);
      return status[i];
    }
  return HM_OK;
}

extern "C" hm_status hm_tune_batched(int32_t nops, const hm_operator* ops, hm_tree* const* trees,
                                     const hm_opts* opts, int32_t format,
                                     const int32_t* candidates, int32_t ncand, void* stream,
                                     int32_t* best, double* ms_out) {
  clear_error();
  if (nops < 1 || !candidates || ncand < 1 || !best) {
    set_error("hm_tune_batched: need nops >= 1, candidates, ncand >= 1 and best");
    return HM_EINVAL;
  }
  for (int32_t c = 0; c < ncand; ++c)
    if (candidates[c] < 1) {
      set_error("hm_tune_batched: every candidate must be >= 1");
      return HM_EINVAL;
    }
  std::vector<hm_handle*> outs((size_t)nops, nullptr);
  auto run = [&](int32_t conc, double* ms) -> hm_status {
    HM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    const auto t0 = std::chrono::steady_clock::now();
    HM_TRY(hm_compress_batched(nops, ops, trees, opts, format, conc, stream, outs.data()));
    const auto t1 = std::chrono::steady_clock::now();
    for (hm_handle*& h : outs) {
      hm_destroy(h);
      h = nullptr;
    }
    if (ms) *ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    return HM_OK;
  };
  HM_TRY(run(candidates[0], nullptr));  // warm-up: operator scales, plans, scratch
  double best_ms = 0.0;
  for (int32_t c = 0; c < ncand; ++c) {
    double ms = 0.0;
    HM_TRY(run(candidates[c], &ms));
    if (ms_out) ms_out[c] = ms;
    if (c == 0 || ms < best_ms) {
      best_ms = ms;
      *best = candidates[c];
    }
  }
  return HM_OK;
}
