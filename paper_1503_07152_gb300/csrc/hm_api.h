// Host-side helpers shared by the entry-point files.
#pragma once

#include "hm_internal.h"

namespace hm {

// A device buffer that only grows; freed with the owner.
struct Workspace {
  void* ptr = nullptr;
  size_t cap = 0;
  hm_status reserve(size_t bytes, cudaStream_t st);
  ~Workspace();
};

hm_status device_alloc(void** p, size_t bytes);

// Bump allocator over one device block (all sub-buffers 256-byte aligned).
// A block is laid out by running the same sequence of take() calls twice: once
// on a measuring arena (base == nullptr) to get the exact size, then on the
// allocated block.  take() past cap returns nullptr and sets `overflow`.
struct Arena {
  unsigned char* base = nullptr;
  size_t off = 0, cap = 0;
  bool overflow = false;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    const size_t at = off;
    off += count * sizeof(T);
    if (base == nullptr) return nullptr;  // measuring
    if (off > cap) {
      overflow = true;
      return nullptr;
    }
    return reinterpret_cast<T*>(base + at);
  }
};

// Allocates one device block for `layout(arena)` and runs the layout on it.
template <typename F>
hm_status arena_alloc(void** block, F&& layout) {
  Arena m;
  layout(m);
  const size_t bytes = m.off + 256;
  HM_TRY(device_alloc(block, bytes));
  Arena a;
  a.base = (unsigned char*)*block;
  a.cap = bytes;
  layout(a);
  if (a.overflow) {
    set_error("internal: device block layout overflow");
    return HM_EUNSUPPORTED;
  }
  return HM_OK;
}

}  // namespace hm

hm_status tree_build(int64_t n, int32_t leaf, hm_tree* t);
hm_status tree_plans(hm_tree* t);
hm_status tree_device(hm_tree* t, cudaStream_t st);
void tree_free(hm_tree* t);
