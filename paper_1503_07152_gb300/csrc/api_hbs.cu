// HBS compression with nested bases (Sec. 4.2, Fig. "A storage efficient
// algorithm for compressing an HBS matrix"), its partial apply (Fig.
// "Application of A^(m) in the HBS framework") and the HBS-ID upward sweep with
// adaptive ranks (Sec. 4.3, Fig. "An algorithm for computing the HBS-ID
// representation").
//
// Storage during the sweep: the long bases of two levels (parents and
// children), per-node short halves U_tau(J_alpha,:) = U_alpha^T U_tau(J_alpha,:)
// (r x r, kept with the child alpha), sibling matrices B_ab (kept with a), and
// the vectors y, z; all sample panels are N x 2r.  The long bases of a level are
// released only after that level's A^T step (the storage-efficient figure
// deletes them after the A step, but the transpose peel of the same level still
// needs them).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hm_hbs.h"
#include "hm_hodlr.h"

using namespace hm;

namespace hm {

constexpr double kEpsScaleId = 0.004;  // ID threshold = 0.004 * tol * max(y | z on level 1)

// Host-built list of small GEMMs launched in one kernel.
template <typename T>
struct Items {
  std::vector<GemmItem> v;
  void add(const T* A, int lda, int ta, const T* B, int ldb, int tb, T* C, int ldc, int m, int n,
           int k) {
    GemmItem it;
    it.A = A; it.B = B; it.C = C;
    it.m = m; it.n = n; it.k = k;
    it.lda = lda; it.ldb = ldb; it.ldc = ldc;
    it.ta = ta; it.tb = tb;
    v.push_back(it);
  }
  hm_status run(GemmItem* dev, size_t cap, T alpha, T beta, cudaStream_t st, bool df = false) {
    if (v.empty()) return HM_OK;
    if (v.size() > cap) {
      set_error("internal: too many batched GEMM items");
      return HM_EUNSUPPORTED;
    }
    HM_CUDA_TRY(cudaMemcpyAsync(dev, v.data(), v.size() * sizeof(GemmItem),
                                cudaMemcpyHostToDevice, st));
    int max_m = 0, max_n = 0, max_k = 0;
    for (const GemmItem& g : v) {
      max_m = std::max(max_m, (int)g.m);
      max_n = std::max(max_n, (int)g.n);
      max_k = std::max(max_k, (int)g.k);
    }
    launch_batched_gemm<T>(dev, (int)v.size(), alpha, beta, st, max_m, max_n, max_k, df);
    v.clear();
    // the pageable source was staged by the copy call; the next batch may reuse dev only
    // after this launch has read it, which stream order guarantees
    return check_launch("batched gemm");
  }
};

// Nested-basis state of one compression or of a finished HBS handle.
template <typename T>
struct HbsState {
  int64_t N = 0;
  int r = 0, L = 0;
  const hm_tree* tree = nullptr;
  T* Ucur = nullptr;  // long bases of the level being peeled (N x r)
  T* Vcur = nullptr;
  T* UsH = nullptr;   // heap-indexed r x r
  T* VsH = nullptr;
  T* Bm = nullptr;
  T* y = nullptr;     // heap-indexed r
  T* z = nullptr;
  T* qhat = nullptr;  // heap-indexed r x w workspace
  T* uhat = nullptr;
  double* partial = nullptr;
  GemmItem* items = nullptr;
  size_t items_cap = 0;
  bool df = false;  // double-float Gram products (HM_A32)
};

// S(:, 0:ncols) += sign * A^(m) X  (transpose: (A^(m))^T), column blocks of <= 128.
template <typename T>
hm_status hbs_partial_apply(HbsState<T>& s, int m, const T* X, int64_t ldx, T* S, int64_t lds,
                            int64_t ncols, int trans, T sign, cudaStream_t st) {
  if (m < 1) return HM_OK;
  const int r = s.r;
  const T* Vout = trans ? s.Ucur : s.Vcur;  // projects the source rows
  const T* Uin = trans ? s.Vcur : s.Ucur;   // expands onto the target rows
  const T* Sout = trans ? s.UsH : s.VsH;    // short halves of the upward pass
  const T* Sin = trans ? s.VsH : s.UsH;     // short halves of the downward pass
  const int64_t rr = (int64_t)r * r;
  const LevelPlan& pm = s.tree->plans[m];
  Items<T> it;
  for (int64_t cb = 0; cb < ncols; cb += 128) {
    const int w = (int)std::min<int64_t>(128, ncols - cb);
    const int64_t rw = (int64_t)r * w;
    T* qh = s.qhat;
    T* uh = s.uhat;
    launch_seg_tn<T>(pm.d_tn, pm.n_tn, pm.d_tn_begin, pm.nnodes, pm.node0, Vout, s.N, 0, 0, r,
                     X + cb * ldx, ldx, 0, 0, w, s.partial, qh + pm.node0 * rw, st, s.df);
    for (int lev = m - 1; lev >= 1; --lev) {
      for (int tau = 1 << lev; tau < (2 << lev); ++tau)
        it.add(Sout + (2 * tau) * rr, r, 1, qh + (2 * tau) * rw, r, 0, qh + tau * rw, r, r, w, r);
      HM_TRY(it.run(s.items, s.items_cap, (T)1, (T)0, st, s.df));
      for (int tau = 1 << lev; tau < (2 << lev); ++tau)
        it.add(Sout + (2 * tau + 1) * rr, r, 1, qh + (2 * tau + 1) * rw, r, 0, qh + tau * rw, r, r,
               w, r);
      HM_TRY(it.run(s.items, s.items_cap, (T)1, (T)1, st, s.df));
    }
    // incoming expansions of the root's children and the downward pass
    for (int lev = 1; lev <= m; ++lev) {
      for (int a = 1 << lev; a < (2 << lev); ++a) {
        if (!trans) it.add(s.Bm + a * rr, r, 0, qh + (a ^ 1) * rw, r, 0, uh + a * rw, r, r, w, r);
        else it.add(s.Bm + (a ^ 1) * rr, r, 1, qh + (a ^ 1) * rw, r, 0, uh + a * rw, r, r, w, r);
      }
      HM_TRY(it.run(s.items, s.items_cap, (T)1, (T)0, st, s.df));
      if (lev >= 2) {
        for (int a = 1 << lev; a < (2 << lev); ++a)
          it.add(Sin + a * rr, r, 0, uh + (a >> 1) * rw, r, 0, uh + a * rw, r, r, w, r);
        HM_TRY(it.run(s.items, s.items_cap, (T)1, (T)1, st, s.df));
      }
    }
    launch_seg_nn<T>(pm.d_nn, pm.n_nn, pm.node0, Uin, s.N, 0, 0, r, uh + pm.node0 * rw, rw, r, 0,
                     S + cb * lds, lds, 0, 0, w, sign, (T)1, st, s.df);
  }
  return check_launch("hbs partial apply");
}

template <typename T>
hm_status compress_hbs_t(Ctx<T>& c, HbsState<T>& s, T* D) {
  const int64_t N = c.N;
  const int r = c.r;
  const int L = c.tree->L;
  const int nmax = (int)c.tree->nmax;
  T* Unext = s.Ucur + N * r;  // two level buffers, swapped by pointer
  T* Vnext = s.Vcur + N * r;
  const int64_t rr = (int64_t)r * r;
  for (int level = 0; level < L; ++level) {
    const int lv = level + 1;
    const LevelPlan& lp = c.tree->plans[lv];
    const int pc = level == 0 ? r : 2 * r;
    mark(c, level, 0, HM_PHASE_SAMPLE);
    HM_TRY(sample_level(c, level));  // X = [Omega_2 | Omega_1], S = A X
    mark(c, level, 0, HM_PHASE_PEEL);
    HM_TRY(hbs_partial_apply(s, level, c.X, N, c.S, N, 2 * r, 0, (T)-1, c.st));
    // Y_loc = [Y(I_a, sample half), U_tau(J_a,:) diag(y_tau)] -> [U_a, y_a] = svd(Y_loc, r)
    mark(c, level, 0, HM_PHASE_BASES);
    launch_gather_sample<T>(c.S, N, c.P, N, N, r, lv, c.tree->d_start, L, c.st);
    if (level > 0)
      launch_gather_parent_scaled<T>(s.Ucur, N, c.P, N, N, r, lv, c.tree->d_start, s.y, r, c.st);
    c.side = 0;
    HM_TRY(panel_svd(c, lv, c.P, pc, 2, r, false, Unext, false, c.rank_tmp));
    mark(c, level, 0, HM_PHASE_BASES);
    launch_node_copy<T, T>(lp.nnodes, lp.node0, c.sig, pc, pc, s.y, r, r, r, 1, 0, c.st);
    if (level > 0)  // U_tau short halves: U_a^T U_tau(J_a, :)
      launch_seg_tn<T>(lp.d_tn, lp.n_tn, lp.d_tn_begin, lp.nnodes, lp.node0, Unext, N, 0, 0, r,
                       s.Ucur, N, 0, 0, r, c.partial, s.UsH + lp.node0 * rr, c.st, s.df);
    launch_scatter_probe<T>(Unext, N, c.X, N, N, r, lv, c.tree->d_start, L, c.st);
    mark(c, level, 1, HM_PHASE_SAMPLE);
    HM_TRY(box(c, 1, c.X, c.S, r));
    HM_TRY(box(c, 1, c.X + N * r, c.S + N * r, r));
    nonfinite_check_launch(c.S, N * 2 * r, sizeof(T) == 8, c.flags_dev, c.st);
    mark(c, level, 1, HM_PHASE_PEEL);
    HM_TRY(hbs_partial_apply(s, level, c.X, N, c.S, N, 2 * r, 1, (T)-1, c.st));
    // Z_loc -> [V_a, b, X] = svd(Z_loc, r); B_ba = X(1:r,:) diag(b) (R2-corrected)
    mark(c, level, 1, HM_PHASE_BASES);
    launch_gather_sample<T>(c.S, N, c.P, N, N, r, lv, c.tree->d_start, L, c.st);
    if (level > 0)
      launch_gather_parent_scaled<T>(s.Vcur, N, c.P, N, N, r, lv, c.tree->d_start, s.z, r, c.st);
    c.side = 1;
    HM_TRY(panel_svd(c, lv, c.P, pc, 2, r, false, Vnext, true, c.rank_tmp));
    mark(c, level, 1, HM_PHASE_BASES);
    launch_node_copy<T, T>(lp.nnodes, lp.node0, c.sig, pc, pc, s.z, r, r, r, 1, 0, c.st);
    launch_node_copy<T, T>(lp.nnodes, lp.node0, c.M, (int64_t)pc * r, pc, s.Bm, rr, r, r, r, 1,
                           c.st);
    if (level > 0)
      launch_seg_tn<T>(lp.d_tn, lp.n_tn, lp.d_tn_begin, lp.nnodes, lp.node0, Vnext, N, 0, 0, r,
                       s.Vcur, N, 0, 0, r, c.partial, s.VsH + lp.node0 * rr, c.st, s.df);
    std::swap(s.Ucur, Unext);
    std::swap(s.Vcur, Vnext);
    c.launches += 12;
    HM_TRY(check_launch("hbs level"));
  }
  mark(c, L, 0, HM_PHASE_SAMPLE);
  HM_TRY(sample_identity(c));
  mark(c, L, 0, HM_PHASE_PEEL);
  HM_TRY(hbs_partial_apply(s, L, c.XI, N, c.YI, N, nmax, 0, (T)-1, c.st));
  mark(c, L, 0, HM_PHASE_BASES);
  launch_extract_diag<T>(c.YI, N, D, nmax, c.tree->d_start, c.tree->d_size, L, c.st);
  return check_launch("hbs diagonal");
}

// ------------------------------------------------------------ HBS-ID -------
// Device layout of an HBS-ID handle (element type T unless noted), heap-indexed:
//   Tin, Tout: r x ncol(node) column-major (ld r); ncol = nmax at leaves, 2r above
//   Bsk: r x r per node (B_skel of the pair (node, sibling))
//   D: leaves x nmax x nmax
//   skel (int64): row / column skeletons, r per node, -1 padded
struct IdLayout {
  int64_t tin_leaf, tin_par, bsk, d;  // element offsets
  int64_t total;
};

template <typename T>
hm_status hbsid_sweep(Ctx<T>& c, HbsState<T>& s, const T* D, hm_handle* h) {
  const int64_t N = c.N;
  const int r = c.r;
  const int L = c.tree->L;
  const int nmax = (int)c.tree->nmax;
  const int nheap = 1 << (L + 1);
  const int nleaf = 1 << L;
  const int64_t rr = (int64_t)r * r;
  cudaStream_t st = c.st;
  // thresholds from the level-1 sample scales (copied to the host once)
  std::vector<T> yz(4 * r);
  HM_CUDA_TRY(cudaMemcpyAsync(yz.data(), s.y + 2 * r, sizeof(T) * 2 * r, cudaMemcpyDeviceToHost, st));
  HM_CUDA_TRY(cudaMemcpyAsync(yz.data() + 2 * r, s.z + 2 * r, sizeof(T) * 2 * r,
                              cudaMemcpyDeviceToHost, st));
  HM_CUDA_TRY(cudaStreamSynchronize(st));
  double ymax = 0, zmax = 0;
  for (int i = 0; i < 2 * r; ++i) {
    ymax = std::max(ymax, (double)yz[i]);
    zmax = std::max(zmax, (double)yz[2 * r + i]);
  }
  const double eps_in = c.mode_tol ? kEpsScaleId * c.tol * ymax : 0.0;
  const double eps_out = c.mode_tol ? kEpsScaleId * c.tol * zmax : 0.0;
  const int kcap = c.mode_tol ? r : std::min(r, c.kfix);
  // FP64 scratch
  const int ncmax = std::max(nmax, 2 * r);
  double *Yt, *Tid, *Us, *Vs, *UsH, *VsH, *Bm, *Utmp, *tmp;
  int32_t *J, *kk;
  auto layout = [&](Arena& a) {
    Yt = a.take<double>((size_t)nleaf * r * ncmax);
    Tid = a.take<double>((size_t)nleaf * r * ncmax);
    Us = a.take<double>((size_t)nheap * rr);
    Vs = a.take<double>((size_t)nheap * rr);
    UsH = a.take<double>((size_t)nheap * rr);
    VsH = a.take<double>((size_t)nheap * rr);
    Bm = a.take<double>((size_t)nheap * rr);
    Utmp = a.take<double>((size_t)(nheap / 2) * 2 * rr);
    tmp = a.take<double>((size_t)(nheap / 2) * rr);
    J = a.take<int32_t>((size_t)nleaf * r);
    kk = a.take<int32_t>((size_t)nleaf);
  };
  void* blk = nullptr;
  HM_TRY(arena_alloc(&blk, layout));
  launch_node_copy<T, double>(nheap, 0, s.UsH, rr, r, UsH, rr, r, r, r, 0, st);
  launch_node_copy<T, double>(nheap, 0, s.VsH, rr, r, VsH, rr, r, r, r, 0, st);
  launch_node_copy<T, double>(nheap, 0, s.Bm, rr, r, Bm, rr, r, r, r, 0, st);
  // handle storage
  IdLayout lay;
  lay.tin_leaf = 0;
  lay.tin_par = (int64_t)nleaf * r * nmax;
  lay.bsk = lay.tin_par + (int64_t)nleaf * r * 2 * r;
  lay.d = lay.bsk + (int64_t)nheap * rr;
  lay.total = lay.d + (int64_t)nleaf * nmax * nmax;
  hm_status stt = device_alloc(&h->hbs_store, sizeof(T) * 2 * (size_t)lay.total);
  if (stt == HM_OK) stt = device_alloc((void**)&h->skel, sizeof(int64_t) * 2 * nheap * (size_t)r);
  if (stt != HM_OK) {
    cudaFree(blk);
    return stt;
  }
  h->hbs_bytes = (int64_t)(sizeof(T) * 2 * lay.total + sizeof(int64_t) * 2 * nheap * r);
  T* store_in = (T*)h->hbs_store;        // Tin / Bsk / D
  T* store_out = store_in + lay.total;   // Tout (Bsk, D unused)
  cudaMemsetAsync(h->hbs_store, 0, sizeof(T) * 2 * (size_t)lay.total, st);
  int64_t* skin = h->skel;
  int64_t* skout = h->skel + (int64_t)nheap * r;
  std::vector<int32_t> kin_all(nheap, 0), kout_all(nheap, 0);
  std::vector<int32_t> kbuf(nleaf);
  Items<double> it;
  for (int side = 0; side < 2; ++side) {
    const T* Bl = side == 0 ? s.Ucur : s.Vcur;
    const T* w = side == 0 ? s.y : s.z;
    double* Samp = side == 0 ? Us : Vs;
    double* Sh = side == 0 ? UsH : VsH;
    int64_t* skel = side == 0 ? skin : skout;
    T* store = side == 0 ? store_in : store_out;
    const double eps = side == 0 ? eps_in : eps_out;
    auto& kall = side == 0 ? kin_all : kout_all;
    // leaves
    launch_id_prep_leaf<T>(Bl, N, c.tree->d_start, c.tree->d_size, L, w, r, Yt, nmax, st);
    launch_pivqr_id(nleaf, Yt, r, nmax, eps, kcap, kk, J, Tid, st, s.df);
    launch_usamp_leaf<T>(Bl, N, c.tree->d_start, L, J, r, Samp, skel, st);
    launch_node_copy<double, T>(nleaf, 0, Tid, (int64_t)r * nmax, r, store + lay.tin_leaf,
                                (int64_t)r * nmax, r, r, nmax, 0, st);
    HM_CUDA_TRY(cudaMemcpyAsync(kbuf.data(), kk, sizeof(int32_t) * nleaf, cudaMemcpyDeviceToHost, st));
    HM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < nleaf; ++i) kall[nleaf + i] = kbuf[i];
    for (int lev = L - 1; lev >= 1; --lev) {
      const int n0 = 1 << lev, nn = 1 << lev;
      // U_tmp = [Usamp_a U_tau(J_a,:); Usamp_b U_tau(J_b,:)]
      for (int t = n0; t < n0 + nn; ++t) {
        double* Ut = Utmp + (int64_t)(t - n0) * 2 * rr;
        it.add(Samp + (2 * t) * rr, r, 0, Sh + (2 * t) * rr, r, 0, Ut, 2 * r, r, r, r);
        it.add(Samp + (2 * t + 1) * rr, r, 0, Sh + (2 * t + 1) * rr, r, 0, Ut + r, 2 * r, r, r, r);
      }
      HM_TRY(it.run((GemmItem*)s.items, s.items_cap, 1.0, 0.0, st, s.df));
      launch_id_prep_parent<T>(nn, n0, Utmp, w, r, Yt, st);
      launch_pivqr_id(nn, Yt, r, 2 * r, eps, kcap, kk, J, Tid, st, s.df);
      launch_usamp_parent(nn, n0, Utmp, J, r, Samp, skel, st);
      launch_node_copy<double, T>(nn, 0, Tid, (int64_t)r * 2 * r, r,
                                  store + lay.tin_par + (int64_t)(n0 - 1) * 2 * rr, 2 * rr, r, r,
                                  2 * r, 0, st);
      HM_CUDA_TRY(cudaMemcpyAsync(kbuf.data(), kk, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, st));
      HM_CUDA_TRY(cudaStreamSynchronize(st));
      for (int i = 0; i < nn; ++i) kall[n0 + i] = kbuf[i];
    }
  }
  // B_skel(a) = Usamp_a B_ab Vsamp_b^T for every node a on levels 1..L
  for (int lv = 1; lv <= L; ++lv) {
    const int n0 = 1 << lv;
    // tmp = Usamp_a B_ab for the level, then Bsk = tmp Vsamp_b^T
    for (int x = n0; x < 2 * n0; ++x)
      it.add(Us + x * rr, r, 0, Bm + x * rr, r, 0, tmp + (int64_t)(x - n0) * rr, r, r, r, r);
    HM_TRY(it.run((GemmItem*)s.items, s.items_cap, 1.0, 0.0, st, s.df));
    for (int x = n0; x < 2 * n0; ++x)
      it.add(tmp + (int64_t)(x - n0) * rr, r, 0, Vs + (x ^ 1) * rr, r, 1, Tid + (int64_t)(x - n0) * rr,
             r, r, r, r);
    HM_TRY(it.run((GemmItem*)s.items, s.items_cap, 1.0, 0.0, st, s.df));
    launch_node_copy<double, T>(n0, n0, Tid, rr, r, store_in + lay.bsk, rr, r, r, r, 0, st);
  }
  cudaMemcpyAsync(store_in + lay.d, D, sizeof(T) * (size_t)nleaf * nmax * nmax,
                  cudaMemcpyDeviceToDevice, st);
  HM_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFree(blk);
  h->kin = kin_all;
  h->kout = kout_all;
  h->tin_off = {lay.tin_leaf, lay.tin_par, lay.bsk, lay.d, lay.total};
  return check_launch("hbs-id sweep");
}

// ------------------------------------------------------------ applies ------
template <typename T>
hm_status hbsid_apply_block(const hm_handle* h, int trans, int w, const T* X, T* Y, T* qh, T* uh,
                            GemmItem* items, size_t cap, cudaStream_t st) {
  const hm_tree* t = &h->tree;
  const int r = h->r;
  const int L = t->L;
  const int nmax = (int)t->nmax;
  const int64_t N = h->n;
  const int64_t rr = (int64_t)r * r, rw = (int64_t)r * w;
  const int64_t total = h->tin_off[4];
  const T* sin = (const T*)h->hbs_store;
  const T* sout = sin + total;
  const T* Tin = trans ? sout : sin;
  const T* Tout = trans ? sin : sout;
  const T* Bsk = sin + h->tin_off[2];
  const T* D = sin + h->tin_off[3];
  auto tcol = [&](const T* base, int node) -> const T* {
    if (node >= (1 << L)) return base + (int64_t)(node - (1 << L)) * r * nmax;
    return base + h->tin_off[1] + (int64_t)(node - 1) * 2 * rr;
  };
  Items<T> it;
  // upward: leaves then parents
  for (int leaf = 1 << L; leaf < (2 << L); ++leaf)
    it.add(tcol(Tout, leaf), r, 0, X + t->start[leaf], N, 0, qh + leaf * rw, r, r, w,
           (int)t->size[leaf]);
  HM_TRY(it.run(items, cap, (T)1, (T)0, st));
  for (int lev = L - 1; lev >= 1; --lev) {
    for (int tau = 1 << lev; tau < (2 << lev); ++tau)
      it.add(tcol(Tout, tau), r, 0, qh + (2 * tau) * rw, r, 0, qh + tau * rw, r, r, w, r);
    HM_TRY(it.run(items, cap, (T)1, (T)0, st));
    for (int tau = 1 << lev; tau < (2 << lev); ++tau)
      it.add(tcol(Tout, tau) + rr, r, 0, qh + (2 * tau + 1) * rw, r, 0, qh + tau * rw, r, r, w, r);
    HM_TRY(it.run(items, cap, (T)1, (T)1, st));
  }
  // sibling interactions and downward pass
  for (int lev = 1; lev <= L; ++lev) {
    for (int a = 1 << lev; a < (2 << lev); ++a) {
      if (!trans) it.add(Bsk + a * rr, r, 0, qh + (a ^ 1) * rw, r, 0, uh + a * rw, r, r, w, r);
      else it.add(Bsk + (a ^ 1) * rr, r, 1, qh + (a ^ 1) * rw, r, 0, uh + a * rw, r, r, w, r);
    }
    HM_TRY(it.run(items, cap, (T)1, (T)0, st));
    if (lev >= 2) {
      for (int a = 1 << lev; a < (2 << lev); ++a) {
        const T* Tp = tcol(Tin, a >> 1) + ((a & 1) ? rr : 0);  // rows of the child's slots
        it.add(Tp, r, 1, uh + (a >> 1) * rw, r, 0, uh + a * rw, r, r, w, r);
      }
      HM_TRY(it.run(items, cap, (T)1, (T)1, st));
    }
  }
  for (int leaf = 1 << L; leaf < (2 << L); ++leaf)
    it.add(tcol(Tin, leaf), r, 1, uh + leaf * rw, r, 0, Y + t->start[leaf], N, (int)t->size[leaf],
           w, r);
  HM_TRY(it.run(items, cap, (T)1, (T)0, st));
  launch_blockdiag_apply<T>(D, nmax, trans, X, N, Y, N, w, t->d_start, t->d_size, L, st);
  return check_launch("hbs-id apply");
}

template <typename T>
hm_status hbs_apply_t(const hm_handle* h, int trans, int64_t ncols, const T* X, int64_t ldx, T* Y,
                      int64_t ldy, cudaStream_t st) {
  const int64_t N = h->n;
  const int r = h->r;
  const int nheap = 1 << (h->L + 1);
  const int64_t cbw = 128;
  const size_t cap = 4 * (size_t)nheap + 16;
  T *qh, *uh, *Xc, *Yc;
  GemmItem* items;
  auto layout = [&](Arena& a) {
    qh = a.take<T>((size_t)nheap * r * cbw);
    uh = a.take<T>((size_t)nheap * r * cbw);
    Xc = a.take<T>(N * cbw);
    Yc = a.take<T>(N * cbw);
    items = a.take<GemmItem>(cap);
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
    launch_copy_cols<T>(X + cb * ldx, ldx, Xc, N, N, w, st);
    if (h->format == HM_FORMAT_HBSID) {
      s = hbsid_apply_block<T>(h, trans, w, Xc, Yc, qh, uh, items, cap, st);
    } else {
      s = HM_EUNSUPPORTED;
      set_error("apply of the plain HBS format is served through HBS-ID handles");
    }
    if (s == HM_OK) launch_copy_cols<T>(Yc, N, Y + cb * ldy, ldy, N, w, st);
  }
  cudaFreeAsync(blk, st);
  if (s != HM_OK) return s;
  return check_launch("hbs apply");
}

template hm_status hbs_apply_t<float>(const hm_handle*, int, int64_t, const float*, int64_t,
                                      float*, int64_t, cudaStream_t);
template hm_status hbs_apply_t<double>(const hm_handle*, int, int64_t, const double*, int64_t,
                                       double*, int64_t, cudaStream_t);

void hbs_free(hm_handle* h) {
  if (h->hbs_store) cudaFree(h->hbs_store);
  h->hbs_store = nullptr;
  if (h->skel) cudaFree(h->skel);
  h->skel = nullptr;
}

}  // namespace hm

template <typename T>
static hm_status compress_hbs_entry(const hm_operator* op, hm_tree* tree, const hm_opts* o,
                                    cudaStream_t user_st, hm_handle** out) {
  const int r = opts_r(o);
  if (r > 64) {
    set_error("hm_compress_hbs: r must be at most 64 (2r-column panels)");
    return HM_EUNSUPPORTED;
  }
  for (int64_t x = (int64_t)1 << tree->L; x < ((int64_t)2 << tree->L); ++x)
    if (tree->size[x] < r) {
      set_error("hm_compress_hbs: every leaf must hold at least r indices");
      return HM_EINVAL;
    }
  hm_handle* h = new hm_handle();
  h->format = HM_FORMAT_HBSID;
  h->prec = o->prec;
  h->n = tree->n;
  h->L = tree->L;
  h->r = r;
  Ctx<T> c;
  c.op = op;
  hm_status s = la_begin(c, o, user_st, true);
  const cudaStream_t st = c.st;  // the compression's stream from here on
  if (s == HM_OK) s = tree_build(tree->n, tree->leaf, &h->tree);
  if (s == HM_OK) s = tree_plans(&h->tree);
  if (s == HM_OK) s = tree_device(&h->tree, st);
  const int64_t N = tree->n;
  const int L = tree->L;
  const int nheap = 1 << (L + 1);
  const int64_t rr = (int64_t)r * r;
  c.tree = &h->tree;
  c.N = N;
  c.r = r;
  c.seed = o->seed;
  c.mode_tol = o->mode_tol;
  c.kfix = o->k;
  c.tol = o->tol;
  c.bf16 = (o->prec != HM_FP64);
  HbsState<T> hs;
  hs.df = sizeof(T) == 8 && o->prec == HM_A32;
  hs.N = N;
  hs.r = r;
  hs.L = L;
  hs.tree = &h->tree;
  void* sblk = nullptr;
  int32_t* rank_block = nullptr;
  T* D = nullptr;
  if (s == HM_OK) s = device_alloc((void**)&rank_block, sizeof(int32_t) * 2 * (size_t)nheap);
  c.rank_dev = rank_block;
  c.rank_tmp = rank_block + nheap;
  if (s == HM_OK) s = ctx_alloc(c, 2 * r, tree->nmax);
  int max_tn = 0;
  for (int lv = 1; lv <= L; ++lv) max_tn = std::max(max_tn, h->tree.plans[lv].n_tn);
  hs.items_cap = 8 * (size_t)nheap + 64;
  auto layout = [&](Arena& a) {
    hs.Ucur = a.take<T>(2 * N * r);
    hs.Vcur = a.take<T>(2 * N * r);
    hs.UsH = a.take<T>(nheap * rr);
    hs.VsH = a.take<T>(nheap * rr);
    hs.Bm = a.take<T>(nheap * rr);
    hs.y = a.take<T>(nheap * r);
    hs.z = a.take<T>(nheap * r);
    hs.qhat = a.take<T>((size_t)nheap * r * 128);
    hs.uhat = a.take<T>((size_t)nheap * r * 128);
    hs.partial = a.take<double>((size_t)max_tn * r * 128);
    hs.items = a.take<GemmItem>(hs.items_cap);
    D = a.take<T>(((size_t)1 << L) * tree->nmax * tree->nmax);
    return a.off;
  };
  size_t sbytes = 0;
  {
    Arena m;
    sbytes = layout(m);
  }
  if (s == HM_OK) s = arena_alloc(&sblk, layout);  // leaves hs.* on the real block
  if (s == HM_OK) cudaMemsetAsync(sblk, 0, sbytes, st);
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  c.profile = profiling_on();
  if (s == HM_OK) {
    cudaEventRecord(t0, st);
    s = compress_hbs_t<T>(c, hs, D);
    if (s == HM_OK) {
      // hbs_partial_apply swaps nothing; after the sweep Ucur/Vcur hold the leaf bases
      mark(c, L, 0, HM_PHASE_ID);
      s = hbsid_sweep<T>(c, hs, D, h);
    }
    mark(c, L, 0, -1);  // end of the last phase
    if (s == HM_OK) s = la_join(c);
    cudaEventRecord(t1, st);
  }
  if (s == HM_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error(std::string("hm_compress_hbs: ") + cudaGetErrorString(e));
      s = HM_ECUDA;
    }
  }
  if (s == HM_OK) s = dense_take_timeout(op);
  int32_t flags[4] = {0, 0, 0, 0};
  if (s == HM_OK) {
    cudaMemcpy(flags, c.flags_dev, sizeof(flags), cudaMemcpyDeviceToHost);
    if (flags[0]) {
      set_error("hm_compress_hbs: NaN or Inf in the black-box samples");
      s = HM_ENONFINITE;
    }
  }
  if (s == HM_OK) {
    hm_info_t& in = h->info;
    std::memset(&in, 0, sizeof(in));
    in.format = HM_FORMAT_HBSID;
    in.prec = o->prec;
    in.n = N;
    in.levels = L;
    in.r = r;
    in.max_rank = 0;
    in.min_rank = r;
    for (int x = 2; x < nheap; ++x) {
      in.max_rank = std::max({in.max_rank, h->kin[x], h->kout[x]});
      in.min_rank = std::min({in.min_rank, h->kin[x], h->kout[x]});
      in.saturated += (h->kin[x] == r) + (h->kout[x] == r);
    }
    in.cols_A = c.cols_A;
    in.cols_At = c.cols_At;
    in.bytes = h->hbs_bytes;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    in.t_compress_ms = ms;
    in.t_blackbox_ms = box_ms(c);
    in.launches = c.launches;
    in.eps_abs = 0.0;
    if (o->strict_rank && in.saturated) {
      set_error("hm_compress_hbs: " + std::to_string(in.saturated) +
                " skeleton ranks reached r (raise r)");
      s = HM_ERANK_SATURATED;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  marks_finish(c, s == HM_OK ? h : nullptr);
  la_end(c);
  ctx_free(c);
  if (rank_block) cudaFree(rank_block);
  if (sblk) cudaFree(sblk);
  if (s != HM_OK) {
    hm_destroy(h);
    return s;
  }
  *out = h;
  return HM_OK;
}

extern "C" hm_status hm_compress_hbs(const hm_operator* op, const hm_tree* tree, const hm_opts* opts,
                                     void* stream, hm_handle** out) {
  clear_error();
  if (!op || !op->apply || !tree || !opts || !out || op->n != tree->n || tree->L < 1 ||
      (opts->prec != HM_FP64 && opts->prec != HM_MIXED && opts->prec != HM_A32)) {
    set_error("hm_compress_hbs: need operator, tree (L >= 1, same n), opts, out");
    return HM_EINVAL;
  }
  if (opts->mode_tol ? !(opts->tol > 0.0 && opts->tol < 1.0) || opts->r < 1
                     : opts->k < 1 || opts->p < 0) {
    set_error("hm_compress_hbs: bad rank / tolerance options");
    return HM_EINVAL;
  }
  if (!opts->hbs_id) {
    set_error("hm_compress_hbs: this library returns HBS-ID handles only (set hbs_id = 1)");
    return HM_EUNSUPPORTED;
  }
  *out = nullptr;
  hm_tree* t = const_cast<hm_tree*>(tree);
  if (opts->prec != HM_MIXED)
    return compress_hbs_entry<double>(op, t, opts, (cudaStream_t)stream, out);
  return compress_hbs_entry<float>(op, t, opts, (cudaStream_t)stream, out);
}
