// Batched compression of independent operators: many operators of uneven size
// and rank compressed in one call.  Each operator's compression is the same
// hot path as hm_compress_hodlr / hm_compress_hbs; the operators run
// concurrently, each on a stream of its own, from a small pool of host threads.
#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "hm_api.h"

using namespace hm;

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
