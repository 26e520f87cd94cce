// Kernels of the HBS / HBS-ID path (Secs. 4.1-4.3):
//  - parent spanning matrix  U_tau(J_alpha,:) diag(y_tau)  appended to a panel
//    (Fig. "A storage efficient algorithm for compressing an HBS matrix"),
//  - batched small GEMMs and per-node copies (short bases, sibling matrices,
//    the upward / downward passes of Fig. "Application of A^(m) in the HBS
//    framework"),
//  - the interpolative decomposition of the HBS-ID sweep (Fig. "An algorithm
//    for computing the HBS-ID representation"): column-pivoted Householder QR
//    (Businger-Golub, largest remaining column norm, lowest index on ties) and
//    T = R11^{-1} [R11 R12] in FP64, one block per node.
#include <atomic>

#include "df.cuh"
#include "hm_internal.h"
#include "hm_hbs.h"

namespace hm {
namespace {

__device__ __forceinline__ int node_of_row_h(const int64_t* __restrict__ start, int lv,
                                             int64_t row) {
  const int64_t* s = start + (1 << lv);
  int lo = 0, hi = (1 << lv) - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s[mid] <= row) lo = mid; else hi = mid - 1;
  }
  return (1 << lv) + lo;
}

// P(i, col0 + j) = U(i, j) * y[parent(node(i))][j]
template <typename T>
__global__ void k_gather_parent_scaled(const T* __restrict__ U, int64_t ldu, T* __restrict__ P,
                                       int64_t ldp, int64_t n, int r, int lv,
                                       const int64_t* __restrict__ start,
                                       const T* __restrict__ y, int col0) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  const int node = node_of_row_h(start, lv, i);
  P[i + (int64_t)(col0 + j) * ldp] = U[i + (int64_t)j * ldu] * y[(int64_t)(node >> 1) * r + j];
}

// C = alpha op(A) op(B) + beta C, one block per item; small sizes.
template <typename T>
__global__ void k_batched_gemm(const GemmItem* __restrict__ items, T alpha, T beta) {
  const GemmItem it = items[blockIdx.x];
  const T* A = (const T*)it.A;
  const T* B = (const T*)it.B;
  T* Cm = (T*)it.C;
  const int mn = it.m * it.n;
  for (int e = threadIdx.x; e < mn; e += blockDim.x) {
    const int i = e % it.m, j = e / it.m;
    T acc = 0;
    for (int p = 0; p < it.k; ++p) {
      const T a = it.ta ? A[p + (int64_t)i * it.lda] : A[i + (int64_t)p * it.lda];
      const T b = it.tb ? B[j + (int64_t)p * it.ldb] : B[p + (int64_t)j * it.ldb];
      acc = fma(a, b, acc);
    }
    T* c = Cm + i + (int64_t)j * it.ldc;
    *c = (beta == (T)0) ? alpha * acc : alpha * acc + beta * (*c);
  }
}

// The same products tiled over blocks: block (item, column tile, row tile)
// computes a 32 x 32 tile of C with its rows of op(A) (32 x k) and its columns of
// op(B) (k x 32) staged in shared memory; thread (i0, j) = (tid / 32, tid % 32)
// keeps rows i0, i0 + 8, i0 + 16, i0 + 24 of column j in registers.  A product's
// FP64 work then spreads over many SMs (the coarse levels have few items, and one
// SM's FP64 rate is low).  Each output is summed over p in the same order as
// k_batched_gemm, so the results are identical.
template <typename T>
__global__ __launch_bounds__(256) void k_batched_gemm_tiled(const GemmItem* __restrict__ items,
                                                            T alpha, T beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GemmItem it = items[blockIdx.x];
  const int m = it.m, n = it.n, k = it.k;
  const int j0 = blockIdx.y * 32, m0 = blockIdx.z * 32;
  if (j0 >= n || m0 >= m) return;  // uniform over the block
  const T* A = (const T*)it.A;
  const T* B = (const T*)it.B;
  T* Cm = (T*)it.C;
  T* As = reinterpret_cast<T*>(smem_raw);  // [32][k]: rows m0 .. m0 + 31 of op(A)
  T* Bs = As + 32 * k;                      // [k][32]: columns j0 .. j0 + 31 of op(B)
  const int tid = threadIdx.x;
  for (int e = tid; e < 32 * k; e += 256) {
    const int ii = e / k, p = e % k, i = m0 + ii;
    As[e] = (i < m) ? (it.ta ? A[p + (int64_t)i * it.lda] : A[i + (int64_t)p * it.lda]) : (T)0;
  }
  for (int e = tid; e < k * 32; e += 256) {
    const int p = e >> 5, col = j0 + (e & 31);
    Bs[e] = (col < n) ? (it.tb ? B[col + (int64_t)p * it.ldb] : B[p + (int64_t)col * it.ldb])
                      : (T)0;
  }
  __syncthreads();
  const int j = tid & 31, i0 = tid >> 5;
  T acc[4] = {0, 0, 0, 0};
  for (int p = 0; p < k; ++p) {
    const T b = Bs[p * 32 + j];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(As[(i0 + 8 * q) * k + p], b, acc[q]);
  }
  const int col = j0 + j;
  if (col < n) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = m0 + i0 + 8 * q;
      if (i < m) {
        T* c = Cm + i + (int64_t)col * it.ldc;
        *c = (beta == (T)0) ? alpha * acc[q] : alpha * acc[q] + beta * (*c);
      }
    }
  }
}

// The FP64 form of k_batched_gemm_tiled in double-float on the FP32 pipe
// (HM_A32): every input cut once, when staged, into hi + lo floats; each output
// summed as a float pair (TwoProduct of the high parts, the cross terms, TwoSum).
__global__ __launch_bounds__(256) void k_batched_gemm_tiled_df(const GemmItem* __restrict__ items,
                                                               double alpha, double beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GemmItem it = items[blockIdx.x];
  const int m = it.m, n = it.n, k = it.k;
  const int j0 = blockIdx.y * 32, m0 = blockIdx.z * 32;
  if (j0 >= n || m0 >= m) return;  // uniform over the block
  const double* A = (const double*)it.A;
  const double* B = (const double*)it.B;
  double* Cm = (double*)it.C;
  float* Ah = reinterpret_cast<float*>(smem_raw);  // [32][k]: rows m0 .. m0 + 31 of op(A)
  float* Al = Ah + 32 * k;
  float* Bh = Al + 32 * k;                         // [k][32]: columns j0 .. j0 + 31 of op(B)
  float* Bl = Bh + 32 * k;
  const int tid = threadIdx.x;
  for (int e = tid; e < 32 * k; e += 256) {
    const int ii = e / k, p = e % k, i = m0 + ii;
    const double v = (i < m) ? (it.ta ? A[p + (int64_t)i * it.lda] : A[i + (int64_t)p * it.lda]) : 0.0;
    df::split(v, Ah[e], Al[e]);
  }
  for (int e = tid; e < k * 32; e += 256) {
    const int p = e >> 5, col = j0 + (e & 31);
    const double v = (col < n) ? (it.tb ? B[col + (int64_t)p * it.ldb] : B[p + (int64_t)col * it.ldb])
                               : 0.0;
    df::split(v, Bh[e], Bl[e]);
  }
  __syncthreads();
  const int j = tid & 31, i0 = tid >> 5;
  float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
  for (int p = 0; p < k; ++p) {
    const float bh = Bh[p * 32 + j], bl = Bl[p * 32 + j];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      df::dot_acc(Ah[(i0 + 8 * q) * k + p], Al[(i0 + 8 * q) * k + p], bh, bl, sh[q], sl[q]);
  }
  const int col = j0 + j;
  if (col < n) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = m0 + i0 + 8 * q;
      if (i < m) {
        double* c = Cm + i + (int64_t)col * it.ldc;
        const double a = df::join(sh[q], sl[q]);
        *c = (beta == 0.0) ? alpha * a : alpha * a + beta * (*c);
      }
    }
  }
}

// dst[(node0 + i) ^ flip] (rows x cols, ld dld) = src[i] (ld sld); heap-indexed dst.
template <typename TS, typename TD>
__global__ void k_node_copy(int node0, const TS* __restrict__ src, int64_t sstride, int sld,
                            TD* __restrict__ dst, int64_t dstride, int dld, int rows, int cols,
                            int flip) {
  const int i = blockIdx.x;
  const int dnode = (node0 + i) ^ flip;
  const TS* s = src + (int64_t)i * sstride;
  TD* d = dst + (int64_t)dnode * dstride;
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    const int rr = e % rows, cc = e / rows;
    d[rr + (int64_t)cc * dld] = (TD)s[rr + (int64_t)cc * sld];
  }
}

// Y_tmp^T of a leaf: Yt(i, j) = y[leaf][i] * U(s + j, i), i < r, j < n_leaf (FP64).
template <typename T>
__global__ void k_id_prep_leaf(const T* __restrict__ U, int64_t ldu,
                               const int64_t* __restrict__ start, const int64_t* __restrict__ size,
                               int L, const T* __restrict__ y, int r, double* __restrict__ Yt,
                               int ncmax) {
  const int leaf = (1 << L) + blockIdx.x;
  const int64_t s = start[leaf];
  const int ns = (int)size[leaf];
  double* Y = Yt + (int64_t)blockIdx.x * r * ncmax;
  for (int e = threadIdx.x; e < r * ncmax; e += blockDim.x) {
    const int i = e % r, j = e / r;
    Y[e] = (j < ns) ? (double)y[(int64_t)leaf * r + i] * (double)U[s + j + (int64_t)i * ldu] : 0.0;
  }
}

// Y_tmp^T of a parent: Yt(i, j) = y[node][i] * Utmp(j, i), Utmp 2r x r per node.
template <typename T>
__global__ void k_id_prep_parent(int node0, const double* __restrict__ Utmp,
                                 const T* __restrict__ y, int r, double* __restrict__ Yt) {
  const int node = node0 + blockIdx.x;
  const double* Ut = Utmp + (int64_t)blockIdx.x * 2 * r * r;
  double* Y = Yt + (int64_t)blockIdx.x * r * 2 * r;
  for (int e = threadIdx.x; e < r * 2 * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    Y[e] = (double)y[(int64_t)node * r + i] * Ut[j + (int64_t)i * 2 * r];
  }
}

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Column ID of the r x nc matrix Yt (per node) with tolerance eps (|R_jj| > eps)
// and at most kcap terms.  Outputs k, J (kcap, -1 padded) and T (kcap x nc,
// column-major, zero rows past k): Yt ~= Yt(:, J) T.
__global__ __launch_bounds__(256) void k_pivqr_id(const double* __restrict__ Yt, int r, int nc,
                                                  double eps, int kcap, int32_t* __restrict__ kout,
                                                  int32_t* __restrict__ Jout,
                                                  double* __restrict__ Tout) {
  // layout stride of J and T rows is r (kcap <= r only caps the rank)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* M = reinterpret_cast<double*>(smem_raw);  // r x nc, column-major
  double* nrm = M + r * nc;                          // nc
  int* perm = reinterpret_cast<int*>(nrm + nc);      // nc
  __shared__ double red[8];
  __shared__ int redi[8];
  __shared__ int sk;
  const double* Y = Yt + (int64_t)blockIdx.x * r * nc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < r * nc; e += blockDim.x) M[e] = Y[e];
  for (int j = tid; j < nc; j += blockDim.x) perm[j] = j;
  __syncthreads();
  const int steps = min(r, nc);
  int k = 0;
  for (int j = 0; j < steps; ++j) {
    // norms of the remaining columns over rows j.. (recomputed: exact pivot rule)
    for (int c = j + warp; c < nc; c += 8) {
      double s = 0.0;
      for (int i = j + lane; i < r; i += 32) s += M[i + c * r] * M[i + c * r];
      s = wsum(s);
      if (lane == 0) nrm[c] = s;
    }
    __syncthreads();
    // argmax, first index on ties
    double best = -1.0;
    int bi = nc;
    for (int c = j + tid; c < nc; c += blockDim.x)
      if (nrm[c] > best || (nrm[c] == best && c < bi)) { best = nrm[c]; bi = c; }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { red[warp] = best; redi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = red[0];
      int i0 = redi[0];
      for (int w = 1; w < 8; ++w)
        if (red[w] > b || (red[w] == b && redi[w] < i0)) { b = red[w]; i0 = redi[w]; }
      sk = (sqrt(b) > eps && j < kcap) ? i0 : -1;
    }
    __syncthreads();
    const int p = sk;
    if (p < 0) break;
    if (p != j) {
      for (int i = tid; i < r; i += blockDim.x) {
        const double t = M[i + j * r];
        M[i + j * r] = M[i + p * r];
        M[i + p * r] = t;
      }
      if (tid == 0) { const int t = perm[j]; perm[j] = perm[p]; perm[p] = t; }
    }
    __syncthreads();
    // Householder on column j (rows j..r-1)
    if (warp == 0) {
      double s = 0.0;
      for (int i = j + lane; i < r; i += 32) s += M[i + j * r] * M[i + j * r];
      s = wsum(s);
      if (lane == 0) {
        const double x0 = M[j + j * r];
        const double nx = sqrt(s);
        const double alpha = (x0 > 0.0) ? -nx : nx;
        const double v0 = x0 - alpha;
        const double vtv = s - x0 * x0 + v0 * v0;
        red[0] = alpha;
        red[1] = (vtv > 0.0) ? 2.0 / vtv : 0.0;
        M[j + j * r] = v0;
      }
    }
    __syncthreads();
    const double beta = red[1];
    for (int c = j + 1 + warp; c < nc; c += 8) {
      double d = 0.0;
      for (int i = j + lane; i < r; i += 32) d += M[i + j * r] * M[i + c * r];
      d = wsum(d) * beta;
      for (int i = j + lane; i < r; i += 32) M[i + c * r] -= d * M[i + j * r];
    }
    __syncthreads();
    if (tid == 0) M[j + j * r] = red[0];
    for (int i = j + 1 + tid; i < r; i += blockDim.x) M[i + j * r] = 0.0;
    __syncthreads();
    k = j + 1;
  }
  // T(:, perm) = [I, R11^{-1} R12]; solve column by column (back substitution)
  double* T = Tout + (int64_t)blockIdx.x * r * nc;
  for (int e = tid; e < r * nc; e += blockDim.x) T[e] = 0.0;
  __syncthreads();
  for (int c = tid; c < nc; c += blockDim.x) {
    const int oc = perm[c];
    if (c < k) {
      T[c + (int64_t)oc * r] = 1.0;
    } else {
      for (int i = k - 1; i >= 0; --i) {
        double s = M[i + c * r];
        for (int q = i + 1; q < k; ++q) s -= M[i + q * r] * T[q + (int64_t)oc * r];
        T[i + (int64_t)oc * r] = s / M[i + i * r];
      }
    }
  }
  int32_t* J = Jout + (int64_t)blockIdx.x * r;
  for (int a = tid; a < r; a += blockDim.x) J[a] = (a < k) ? perm[a] : -1;
  if (tid == 0) kout[blockIdx.x] = k;
}

// k_pivqr_id in double-float (HM_A32): the same column-pivoted Householder QR
// with the exact pivot rule (norms recomputed each step, the largest first,
// the first index on ties) and T = R11^{-1} R12 by back substitution, with every
// operation carried by float pairs on the FP32 pipe (FP64 in and out).  The
// columns of R12 are overwritten by T in place during the substitution.
__global__ __launch_bounds__(256) void k_pivqr_id_df(const double* __restrict__ Yt, int r, int nc,
                                                     double eps, int kcap,
                                                     int32_t* __restrict__ kout,
                                                     int32_t* __restrict__ Jout,
                                                     double* __restrict__ Tout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Mh = reinterpret_cast<float*>(smem_raw);  // r x nc, column-major
  float* Ml = Mh + (size_t)r * nc;
  float* nh = Ml + (size_t)r * nc;                 // nc: squared norms (pairs)
  float* nl = nh + nc;
  int* perm = reinterpret_cast<int*>(nl + nc);     // nc
  __shared__ float redh[8], redl[8], sh_a[2], sh_b[2];
  __shared__ int redi[8];
  __shared__ int sk;
  const double* Y = Yt + (int64_t)blockIdx.x * r * nc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < r * nc; e += blockDim.x) df::split(Y[e], Mh[e], Ml[e]);
  for (int j = tid; j < nc; j += blockDim.x) perm[j] = j;
  // eps^2 as a pair, for the rank test |col|^2 > eps^2
  float e2h, e2l;
  df::split(eps * eps, e2h, e2l);
  __syncthreads();
  const int steps = min(r, nc);
  int k = 0;
  for (int j = 0; j < steps; ++j) {
    for (int c = j + warp; c < nc; c += 8) {
      float s = 0.f, t = 0.f;
      for (int i = j + lane; i < r; i += 32)
        df::dot_acc(Mh[i + c * r], Ml[i + c * r], Mh[i + c * r], Ml[i + c * r], s, t);
      df::warp_sum(s, t);
      if (lane == 0) df::fast_two_sum(s, t, nh[c], nl[c]);
    }
    __syncthreads();
    float bh = -1.f, bl = 0.f;
    int bi = nc;
    for (int c = j + tid; c < nc; c += blockDim.x)
      if (nh[c] > bh || (nh[c] == bh && nl[c] > bl)) { bh = nh[c]; bl = nl[c]; bi = c; }
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, bh, o);
      const float ol = __shfl_xor_sync(0xffffffffu, bl, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oh > bh || (oh == bh && (ol > bl || (ol == bl && oi < bi)))) { bh = oh; bl = ol; bi = oi; }
    }
    if (lane == 0) { redh[warp] = bh; redl[warp] = bl; redi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      float b = redh[0], bb = redl[0];
      int i0 = redi[0];
      for (int w = 1; w < 8; ++w)
        if (redh[w] > b || (redh[w] == b && (redl[w] > bb || (redl[w] == bb && redi[w] < i0)))) {
          b = redh[w]; bb = redl[w]; i0 = redi[w];
        }
      const bool above = b > e2h || (b == e2h && bb > e2l);
      sk = (above && j < kcap) ? i0 : -1;
    }
    __syncthreads();
    const int p = sk;
    if (p < 0) break;
    if (p != j) {
      for (int i = tid; i < r; i += blockDim.x) {
        float t = Mh[i + j * r]; Mh[i + j * r] = Mh[i + p * r]; Mh[i + p * r] = t;
        t = Ml[i + j * r]; Ml[i + j * r] = Ml[i + p * r]; Ml[i + p * r] = t;
      }
      if (tid == 0) { const int t = perm[j]; perm[j] = perm[p]; perm[p] = t; }
    }
    __syncthreads();
    // Householder on column j (rows j..r-1)
    if (warp == 0) {
      float s = 0.f, t = 0.f;
      for (int i = j + lane; i < r; i += 32)
        df::dot_acc(Mh[i + j * r], Ml[i + j * r], Mh[i + j * r], Ml[i + j * r], s, t);
      df::warp_sum(s, t);
      if (lane == 0) {
        const float xh = Mh[j + j * r], xl = Ml[j + j * r];
        float nxh, nxl;
        df::sqrt_df(s, t, nxh, nxl);
        const float ah = (xh > 0.f) ? -nxh : nxh, al = (xh > 0.f) ? -nxl : nxl;
        float vh, vl, wh = nxh, wl = nxl, qh, ql;
        df::sub(xh, xl, ah, al, vh, vl);                    // v0 = x0 - alpha
        df::add_to(wh, wl, fabsf(xh), xh < 0.f ? -xl : xl);  // nrm + |x0|
        df::mul(nxh, nxl, wh, wl, qh, ql);                   // v^T v / 2
        sh_a[0] = ah;
        sh_a[1] = al;
        if (qh > 0.f) {
          df::div_df(1.f, 0.f, qh, ql, sh_b[0], sh_b[1]);   // beta = 2 / v^T v
        } else {
          sh_b[0] = 0.f;
          sh_b[1] = 0.f;
        }
        Mh[j + j * r] = vh;
        Ml[j + j * r] = vl;
      }
    }
    __syncthreads();
    const float beh = sh_b[0], bel = sh_b[1];
    for (int c = j + 1 + warp; c < nc; c += 8) {
      float dh = 0.f, dl = 0.f;
      for (int i = j + lane; i < r; i += 32)
        df::dot_acc(Mh[i + j * r], Ml[i + j * r], Mh[i + c * r], Ml[i + c * r], dh, dl);
      df::warp_sum(dh, dl);
      float fh, fl;
      df::mul(dh, dl, beh, bel, fh, fl);
      for (int i = j + lane; i < r; i += 32)
        df::axpy_neg(fh, fl, Mh[i + j * r], Ml[i + j * r], Mh[i + c * r], Ml[i + c * r]);
    }
    __syncthreads();
    if (tid == 0) { Mh[j + j * r] = sh_a[0]; Ml[j + j * r] = sh_a[1]; }
    for (int i = j + 1 + tid; i < r; i += blockDim.x) { Mh[i + j * r] = 0.f; Ml[i + j * r] = 0.f; }
    __syncthreads();
    k = j + 1;
  }
  // inverse diagonal of R11, then T(:, perm) = [I, R11^{-1} R12] column by column
  // (back substitution; column c's T overwrites its R12 entries as they are used)
  for (int i = tid; i < k; i += blockDim.x) df::div_df(1.f, 0.f, Mh[i + i * r], Ml[i + i * r], nh[i], nl[i]);
  __syncthreads();
  double* T = Tout + (int64_t)blockIdx.x * r * nc;
  for (int e = tid; e < r * nc; e += blockDim.x) T[e] = 0.0;
  __syncthreads();
  for (int c = tid; c < nc; c += blockDim.x) {
    const int oc = perm[c];
    if (c < k) {
      T[c + (int64_t)oc * r] = 1.0;
    } else {
      for (int i = k - 1; i >= 0; --i) {
        float sh = Mh[i + c * r], sl = Ml[i + c * r];
        for (int q = i + 1; q < k; ++q)
          df::axpy_neg(Mh[q + c * r], Ml[q + c * r], Mh[i + q * r], Ml[i + q * r], sh, sl);
        df::mul(sh, sl, nh[i], nl[i], Mh[i + c * r], Ml[i + c * r]);
      }
      for (int i = 0; i < k; ++i) T[i + (int64_t)oc * r] = df::join(Mh[i + c * r], Ml[i + c * r]);
    }
  }
  int32_t* J = Jout + (int64_t)blockIdx.x * r;
  for (int a = tid; a < r; a += blockDim.x) J[a] = (a < k) ? perm[a] : -1;
  if (tid == 0) kout[blockIdx.x] = k;
}

// Usamp (r x r, row a = skeleton row a, zero rows past k) from a leaf basis.
template <typename T>
__global__ void k_usamp_leaf(const T* __restrict__ U, int64_t ldu, const int64_t* __restrict__ start,
                             int L, const int32_t* __restrict__ J, int r,
                             double* __restrict__ Us, int64_t* __restrict__ skel) {
  const int leaf = (1 << L) + blockIdx.x;
  const int64_t s = start[leaf];
  const int32_t* Jl = J + (int64_t)blockIdx.x * r;
  double* Ul = Us + (int64_t)leaf * r * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e % r, c = e / r;
    const int ja = Jl[a];
    Ul[e] = (ja >= 0) ? (double)U[s + ja + (int64_t)c * ldu] : 0.0;
  }
  for (int a = threadIdx.x; a < r; a += blockDim.x)
    skel[(int64_t)leaf * r + a] = (Jl[a] >= 0) ? s + Jl[a] : -1;
}

// Parent: Usamp = Utmp(J, :) and skeleton = children's skeletons at J.
__global__ void k_usamp_parent(int node0, const double* __restrict__ Utmp,
                               const int32_t* __restrict__ J, int r, double* __restrict__ Us,
                               int64_t* __restrict__ skel) {
  const int node = node0 + blockIdx.x;
  const double* Ut = Utmp + (int64_t)blockIdx.x * 2 * r * r;
  const int32_t* Jn = J + (int64_t)blockIdx.x * r;
  double* Un = Us + (int64_t)node * r * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e % r, c = e / r;
    const int ja = Jn[a];
    Un[e] = (ja >= 0) ? Ut[ja + (int64_t)c * 2 * r] : 0.0;
  }
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    const int ja = Jn[a];
    int64_t g = -1;
    if (ja >= 0) g = (ja < r) ? skel[(int64_t)(2 * node) * r + ja] : skel[(int64_t)(2 * node + 1) * r + ja - r];
    skel[(int64_t)node * r + a] = g;
  }
}

}  // namespace

template <typename T>
void launch_gather_parent_scaled(const T* U, int64_t ldu, T* P, int64_t ldp, int64_t n, int r,
                                 int lv, const int64_t* d_start, const T* y, int col0,
                                 cudaStream_t st) {
  count_launches(1);
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)r);
  k_gather_parent_scaled<T><<<grid, 256, 0, st>>>(U, ldu, P, ldp, n, r, lv, d_start, y, col0);
}

template <typename T>
void launch_batched_gemm(const GemmItem* items, int count, T alpha, T beta, cudaStream_t st,
                         int max_m, int max_n, int max_k, bool df) {
  if (count <= 0) return;
  count_launches(1);
  const size_t smem = (size_t)64 * max_k * sizeof(T);
  if (max_m >= 1 && max_n >= 1 && max_k >= 1 && smem <= 96 * 1024 && max_n <= 32 * 65535 &&
      max_m <= 32 * 65535 && sizeof(T) == 8 && df) {
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_batched_gemm_tiled_df, done);
    dim3 grid((unsigned)count, (unsigned)((max_n + 31) / 32), (unsigned)((max_m + 31) / 32));
    k_batched_gemm_tiled_df<<<grid, 256, smem, st>>>(items, (double)alpha, (double)beta);
  } else if (max_m >= 1 && max_n >= 1 && max_k >= 1 && smem <= 96 * 1024 &&
             max_n <= 32 * 65535 && max_m <= 32 * 65535) {
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_batched_gemm_tiled<T>, done);
    dim3 grid((unsigned)count, (unsigned)((max_n + 31) / 32), (unsigned)((max_m + 31) / 32));
    k_batched_gemm_tiled<T><<<grid, 256, smem, st>>>(items, alpha, beta);
  } else {
    k_batched_gemm<T><<<count, 256, 0, st>>>(items, alpha, beta);
  }
}

template <typename TS, typename TD>
void launch_node_copy(int nnodes, int node0, const TS* src, int64_t sstride, int sld, TD* dst,
                      int64_t dstride, int dld, int rows, int cols, int flip, cudaStream_t st) {
  if (nnodes <= 0) return;
  count_launches(1);
  k_node_copy<TS, TD><<<nnodes, 256, 0, st>>>(node0, src, sstride, sld, dst, dstride, dld, rows,
                                              cols, flip);
}

template <typename T>
void launch_id_prep_leaf(const T* U, int64_t ldu, const int64_t* d_start, const int64_t* d_size,
                         int L, const T* y, int r, double* Yt, int ncmax, cudaStream_t st) {
  count_launches(1);
  k_id_prep_leaf<T><<<1 << L, 256, 0, st>>>(U, ldu, d_start, d_size, L, y, r, Yt, ncmax);
}

template <typename T>
void launch_id_prep_parent(int nnodes, int node0, const double* Utmp, const T* y, int r,
                           double* Yt, cudaStream_t st) {
  count_launches(1);
  k_id_prep_parent<T><<<nnodes, 256, 0, st>>>(node0, Utmp, y, r, Yt);
}

void launch_pivqr_id(int nnodes, const double* Yt, int r, int nc, double eps, int kcap,
                     int32_t* k, int32_t* J, double* T, cudaStream_t st, bool df) {
  count_launches(1);
  const size_t smem = sizeof(double) * ((size_t)r * nc + nc) + sizeof(int) * nc;
  if (df) {  // the same layout size: float pairs in place of doubles
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_pivqr_id_df, done);
    k_pivqr_id_df<<<nnodes, 256, smem, st>>>(Yt, r, nc, eps, kcap, k, J, T);
    return;
  }
  static std::atomic<uint32_t> done{0};
  raise_smem_limit((const void*)k_pivqr_id, done);
  k_pivqr_id<<<nnodes, 256, smem, st>>>(Yt, r, nc, eps, kcap, k, J, T);
}

template <typename T>
void launch_usamp_leaf(const T* U, int64_t ldu, const int64_t* d_start, int L, const int32_t* J,
                       int r, double* Us, int64_t* skel, cudaStream_t st) {
  count_launches(1);
  k_usamp_leaf<T><<<1 << L, 128, 0, st>>>(U, ldu, d_start, L, J, r, Us, skel);
}

void launch_usamp_parent(int nnodes, int node0, const double* Utmp, const int32_t* J, int r,
                         double* Us, int64_t* skel, cudaStream_t st) {
  count_launches(1);
  k_usamp_parent<<<nnodes, 128, 0, st>>>(node0, Utmp, J, r, Us, skel);
}

#define HM_INST(T)                                                                             \
  template void launch_gather_parent_scaled<T>(const T*, int64_t, T*, int64_t, int64_t, int,   \
                                               int, const int64_t*, const T*, int,             \
                                               cudaStream_t);                                  \
  template void launch_batched_gemm<T>(const GemmItem*, int, T, T, cudaStream_t, int, int, int, \
                                       bool);              \
  template void launch_id_prep_leaf<T>(const T*, int64_t, const int64_t*, const int64_t*, int, \
                                       const T*, int, double*, int, cudaStream_t);             \
  template void launch_id_prep_parent<T>(int, int, const double*, const T*, int, double*,      \
                                         cudaStream_t);                                        \
  template void launch_usamp_leaf<T>(const T*, int64_t, const int64_t*, int, const int32_t*,   \
                                     int, double*, int64_t*, cudaStream_t);
HM_INST(float)
HM_INST(double)
#undef HM_INST
template void launch_node_copy<float, float>(int, int, const float*, int64_t, int, float*, int64_t,
                                             int, int, int, int, cudaStream_t);
template void launch_node_copy<double, double>(int, int, const double*, int64_t, int, double*,
                                               int64_t, int, int, int, int, cudaStream_t);
template void launch_node_copy<float, double>(int, int, const float*, int64_t, int, double*,
                                              int64_t, int, int, int, int, cudaStream_t);
template void launch_node_copy<double, float>(int, int, const double*, int64_t, int, float*,
                                              int64_t, int, int, int, int, cudaStream_t);

}  // namespace hm
