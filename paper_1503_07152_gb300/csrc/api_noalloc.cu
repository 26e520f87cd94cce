// Factored HODLR apply that allocates no device memory per call: its scratch
// (the per-chunk partial projections and the per-node coefficients of the
// product) lives in a fixed-size buffer compiled into the library instead of
// being taken from the CUDA memory pool.  The kernels are the ones of
// hm_hodlr_factored_apply.
#include <mutex>
#include <string>

#include "hm_internal.h"

using namespace hm;

namespace {

// 8 MiB on every device where the library's device code is loaded.
constexpr size_t kNoallocScratchBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Address of the buffer per device ordinal, looked up on the first call made
// with that device current and kept for the life of the process (a
// cudaDeviceReset of that device invalidates it).
constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" hm_status hm_hodlr_factored_apply_noalloc(const hm_tree* tree, int32_t k,
                                                     const float* U, const float* V,
                                                     const float* D, int trans, const float* x,
                                                     float* y, void* stream) {
  clear_error();
  if (!tree || k < 1 || k > 64 || !U || !V || !D || !x || !y || tree->L < 1 ||
      (trans != 0 && trans != 1)) {
    set_error("hm_hodlr_factored_apply_noalloc: need tree (L >= 1), 1 <= k <= 64, U, V, D, x, y");
    return HM_EINVAL;
  }
  // partial projections (one row of k per 256-row chunk of every node) and the
  // coefficients (k per node), as laid out by the shared launcher
  // (hm_tree_create builds the chunk list, so n_fchunks is exact here)
  const size_t nodes = (size_t)1 << (tree->L + 1);
  const size_t chunks = (size_t)tree->n_fchunks;
  const size_t need = sizeof(float) * (chunks * (size_t)k + nodes * (size_t)k);
  if (need > kNoallocScratchBytes) {
    set_error("hm_hodlr_factored_apply_noalloc: this tree and k need " + std::to_string(need) +
              " bytes of scratch; the static buffer holds " +
              std::to_string(kNoallocScratchBytes) + " (use hm_hodlr_factored_apply)");
    return HM_EINVAL;
  }
  if (!tree->d_start || !tree->d_fchunks || !tree->d_fbegin) {
    set_error(
        "hm_hodlr_factored_apply_noalloc: the tree's index tables are not on the device yet "
        "(uploading them allocates); one call of hm_hodlr_factored_apply with this tree "
        "uploads them");
    return HM_EINVAL;
  }
  int dev = -1;
  HM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("hm_hodlr_factored_apply_noalloc: device ordinal out of range");
    return HM_EINVAL;
  }
  if (tree->dev != dev) {
    set_error("hm_hodlr_factored_apply_noalloc: the tree's index tables were uploaded to device " +
              std::to_string(tree->dev) + ", but device " + std::to_string(dev) + " is current");
    return HM_EINVAL;
  }
  HM_TRY(factored_check(tree, false));
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        (void)cudaGetLastError();
        set_error(std::string("hm_hodlr_factored_apply_noalloc: cudaGetSymbolAddress: ") +
                  cudaGetErrorString(e));
        return HM_ECUDA;
      }
      g_addr[dev] = p;
    }
    scratch = g_addr[dev];
  }
  launch_factored_apply(tree, k, U, V, D, trans, x, y, (float*)scratch, (cudaStream_t)stream);
  return check_launch("hm_hodlr_factored_apply_noalloc");
}
