// Checkpoint of compressed handles: hm_save writes a handle's representation to
// a file (host copies of its device arrays behind a small header and a
// checksum), hm_load rebuilds an equivalent handle on the current device.  The
// solver factors of hm_hodlr_factorize are not stored (factorize again).
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hm_api.h"

using namespace hm;

namespace {

constexpr char kMagic[8] = {'H', 'M', 'C', 'K', 'P', 'T', '0', '1'};

struct Header {
  char magic[8];
  int32_t format, prec;
  int64_t n;
  int32_t leaf, L, r, pad;
  int64_t elem;      // bytes per element (8 double, 4 float)
  int64_t payload;   // bytes after the header
  uint64_t checksum; // FNV-1a over the payload
  hm_info_t info;
};

uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 1469598103934665603ull) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct Blob {
  std::vector<unsigned char> b;
  void put(const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    b.insert(b.end(), c, c + n);
  }
  hm_status put_dev(const void* d, size_t n) {
    const size_t o = b.size();
    b.resize(o + n);
    if (n && cudaMemcpy(b.data() + o, d, n, cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_error("hm_save: device copy failed");
      return HM_ECUDA;
    }
    return HM_OK;
  }
};

struct Reader {
  const unsigned char* p;
  size_t n, off = 0;
  bool get(void* dst, size_t k) {
    if (off + k > n) return false;
    std::memcpy(dst, p + off, k);
    off += k;
    return true;
  }
  const unsigned char* take(size_t k) {
    if (off + k > n) return nullptr;
    const unsigned char* q = p + off;
    off += k;
    return q;
  }
};

}  // namespace

extern "C" hm_status hm_save(const hm_handle* h, const char* path) {
  clear_error();
  if (!h || !path || (h->format != HM_FORMAT_HODLR && h->format != HM_FORMAT_HBSID)) {
    set_error("hm_save: need a HODLR or HBS-ID handle and a path");
    return HM_EINVAL;
  }
  HM_CUDA_TRY(cudaDeviceSynchronize());
  const int64_t es = h->prec == HM_MIXED ? 4 : 8;
  const int64_t N = h->n, r = h->r, L = h->L;
  const int64_t nheap = (int64_t)1 << (L + 1), nleaf = (int64_t)1 << L, nmax = h->tree.nmax;
  Blob body;
  if (h->format == HM_FORMAT_HODLR) {
    body.put(h->rank.data(), sizeof(int32_t) * (size_t)nheap);
    HM_TRY(body.put_dev(h->U, (size_t)(es * L * N * r)));
    HM_TRY(body.put_dev(h->V, (size_t)(es * L * N * r)));
    HM_TRY(body.put_dev(h->D, (size_t)(es * nleaf * nmax * nmax)));
  } else {
    body.put(h->kin.data(), sizeof(int32_t) * (size_t)nheap);
    body.put(h->kout.data(), sizeof(int32_t) * (size_t)nheap);
    body.put(h->tin_off.data(), sizeof(int64_t) * 5);
    HM_TRY(body.put_dev(h->hbs_store, (size_t)(es * 2 * h->tin_off[4])));
    HM_TRY(body.put_dev(h->skel, sizeof(int64_t) * (size_t)(2 * nheap * r)));
  }
  Header hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kMagic, 8);
  hd.format = h->format;
  hd.prec = h->prec;
  hd.n = N;
  hd.leaf = h->tree.leaf;
  hd.L = (int32_t)L;
  hd.r = (int32_t)r;
  hd.elem = es;
  hd.payload = (int64_t)body.b.size();
  hd.checksum = fnv1a(body.b.data(), body.b.size());
  hd.info = h->info;
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    set_error(std::string("hm_save: cannot open ") + path);
    return HM_EINVAL;
  }
  const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
                  (body.b.empty() || std::fwrite(body.b.data(), body.b.size(), 1, f) == 1);
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) {
    set_error(std::string("hm_save: write to ") + path + " failed");
    return HM_EINVAL;
  }
  return HM_OK;
}

extern "C" hm_status hm_load(const char* path, void* stream, hm_handle** out) {
  clear_error();
  if (!path || !out) {
    set_error("hm_load: need a path and out");
    return HM_EINVAL;
  }
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error(std::string("hm_load: cannot open ") + path);
    return HM_EINVAL;
  }
  Header hd;
  std::vector<unsigned char> body;
  bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, kMagic, 8) == 0 &&
            hd.payload >= 0 && hd.payload < ((int64_t)1 << 40);
  if (ok) {
    body.resize((size_t)hd.payload);
    ok = hd.payload == 0 || std::fread(body.data(), body.size(), 1, f) == 1;
  }
  std::fclose(f);
  if (!ok || fnv1a(body.data(), body.size()) != hd.checksum ||
      (hd.format != HM_FORMAT_HODLR && hd.format != HM_FORMAT_HBSID) || hd.n < 1 ||
      hd.leaf < 1 || hd.r < 1 || hd.elem != (hd.prec == HM_MIXED ? 4 : 8)) {
    set_error(std::string("hm_load: ") + path + " is not a valid checkpoint (bad header, size or "
              "checksum)");
    return HM_EINVAL;
  }
  hm_handle* h = new hm_handle();
  h->format = hd.format;
  h->prec = hd.prec;
  h->n = hd.n;
  h->r = hd.r;
  hm_status s = tree_build(hd.n, hd.leaf, &h->tree);
  if (s == HM_OK && h->tree.L != hd.L) {
    set_error("hm_load: tree depth differs from the checkpoint's");
    s = HM_EINVAL;
  }
  h->L = h->tree.L;
  if (s == HM_OK) s = tree_plans(&h->tree);
  if (s == HM_OK) s = tree_device(&h->tree, (cudaStream_t)stream);
  const int64_t es = hd.elem, N = hd.n, r = hd.r, L = h->L;
  const int64_t nheap = (int64_t)1 << (L + 1), nleaf = (int64_t)1 << L, nmax = h->tree.nmax;
  Reader rd{body.data(), body.size()};
  auto to_dev = [&](void** dst, size_t bytes) -> hm_status {
    const unsigned char* src = rd.take(bytes);
    if (!src) {
      set_error("hm_load: checkpoint payload too short");
      return HM_EINVAL;
    }
    HM_TRY(device_alloc(dst, bytes));
    HM_CUDA_TRY(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return HM_OK;
  };
  if (s == HM_OK && hd.format == HM_FORMAT_HODLR) {
    h->rank.assign((size_t)nheap, 0);
    if (!rd.get(h->rank.data(), sizeof(int32_t) * (size_t)nheap)) s = HM_EINVAL;
    if (s == HM_OK) s = to_dev(&h->U, (size_t)(es * L * N * r));
    if (s == HM_OK) s = to_dev(&h->V, (size_t)(es * L * N * r));
    if (s == HM_OK) s = to_dev(&h->D, (size_t)(es * nleaf * nmax * nmax));
  } else if (s == HM_OK) {
    h->kin.assign((size_t)nheap, 0);
    h->kout.assign((size_t)nheap, 0);
    h->tin_off.assign(5, 0);
    if (!rd.get(h->kin.data(), sizeof(int32_t) * (size_t)nheap) ||
        !rd.get(h->kout.data(), sizeof(int32_t) * (size_t)nheap) ||
        !rd.get(h->tin_off.data(), sizeof(int64_t) * 5) || h->tin_off[4] < 0)
      s = HM_EINVAL;
    if (s == HM_OK) s = to_dev(&h->hbs_store, (size_t)(es * 2 * h->tin_off[4]));
    if (s == HM_OK) s = to_dev((void**)&h->skel, sizeof(int64_t) * (size_t)(2 * nheap * r));
    h->hbs_bytes = es * 2 * h->tin_off[4] + (int64_t)sizeof(int64_t) * 2 * nheap * r;
  }
  if (s == HM_OK && rd.off != rd.n) {
    set_error("hm_load: checkpoint payload has trailing bytes");
    s = HM_EINVAL;
  }
  if (s != HM_OK) {
    if (s == HM_EINVAL && !*hm_last_error()) set_error("hm_load: checkpoint payload too short");
    hm_destroy(h);
    return s;
  }
  h->info = hd.info;
  *out = h;
  return HM_OK;
}
