// Per-node orthonormalization and truncated SVD of sample panels, batched over
// all nodes of a level (uneven sizes in one launch):
//   1. TSQR: Householder QR of row blocks of at most 128 rows in shared memory;
//      the R factors are merged pairwise in a tree by a Householder QR of the
//      stacked pair that keeps both triangles packed (R only; Q is never formed).
//   2. SVD of each node's final R.  FP64: a column-pivoted QR R P = Q2 R2
//      (Businger-Golub), then one-sided (Hestenes) Jacobi on X = R2^T, run in
//      FP32 first and finished in FP64 (see k_jacobi_mp).  The normalized
//      rotated columns of X are its left singular vectors U_x, so the right
//      singular vectors of R are W = P U_x and no rotation has to be
//      accumulated; R2^T has graded columns, so the sweeps converge quickly and
//      the small singular values keep their relative accuracy.  FP32: one-sided
//      Jacobi on R with the rotations accumulated into W (orthonormal to
//      working precision, which FP32 needs).  Sorted descending, with a fixed
//      sign convention.
//   3. Truncation: the rank k of the node (mode 2 fixed k, or mode 3 tolerance,
//      Sec. 2.6) and T1 = W(:, :k) S^{-1}, so that Q1 = P T1 has orthonormal
//      columns in exact arithmetic (the left singular vectors of P).
//   4. CholQR pass: Q = Q1 R2^{-1} with R2 = chol(Q1^T Q1) restores
//      orthonormality lost to rounding; the coefficient M = W_k S_k R2^T gives
//      P ~= Q M^T for the sibling matrices (Remark 4 / the svd steps of the
//      HODLR and HBS figures).
// These realize qr(.) and svd(., k | eps) of Secs. 2.2-2.3 / 2.6 for panels too
// tall for one block.
#include <algorithm>

#include "hm_internal.h"

namespace hm {
namespace {

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 5.960464477539063e-08; };
template <> struct Eps<double> { static constexpr double v = 1.1102230246251565e-16; };

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Householder QR of the stacked sources of one task; writes the c x c R
// (row-major, upper triangle, zero rows past min(m, c)).
template <typename T>
__global__ __launch_bounds__(256) void k_tsqr(const TsqrTask* __restrict__ tasks,
                                              const T* __restrict__ P, int64_t ldp, int c,
                                              T* __restrict__ R, int ldm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* M = reinterpret_cast<T*>(smem_raw);  // column-major, ld = ldm
  __shared__ double red[8];
  __shared__ T sh_alpha, sh_beta;
  const TsqrTask tk = tasks[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int m = 0;
  for (int s = 0; s < tk.nsrc; ++s) {
    if (tk.kind[s] == 0) {
      const int rows = (int)(tk.r1[s] - tk.r0[s]);
      for (int idx = tid; idx < rows * c; idx += 256) {
        const int rr = idx % rows, col = idx / rows;
        M[col * ldm + m + rr] = P[tk.r0[s] + rr + (int64_t)col * ldp];
      }
      m += rows;
    } else {
      const T* Rs = R + (int64_t)tk.slot[s] * c * c;
      for (int idx = tid; idx < c * c; idx += 256) {
        const int rr = idx / c, col = idx % c;
        M[col * ldm + m + rr] = Rs[rr * c + col];
      }
      m += c;
    }
  }
  __syncthreads();
  const int steps = m < c ? m : c;
  for (int j = 0; j < steps; ++j) {
    T* mj = M + j * ldm;
    T s = 0;
    for (int i = j + tid; i < m; i += 256) s = fma(mj[i], mj[i], s);
    s = warp_sum(s);
    if (lane == 0) red[warp] = (double)s;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < 8; ++w) tot += red[w];
      const double x0 = (double)mj[j];
      const double nrm = sqrt(tot);
      const double alpha = (x0 > 0.0) ? -nrm : nrm;
      const double v0 = x0 - alpha;
      const double vtv = tot - x0 * x0 + v0 * v0;
      sh_alpha = (T)alpha;
      sh_beta = (vtv > 0.0) ? (T)(2.0 / vtv) : (T)0;
      mj[j] = (T)v0;
    }
    __syncthreads();
    const T beta = sh_beta;
    if (beta != (T)0) {
      // one aligned 8-lane group per trailing column, 32 columns per round
      for (int k0 = j + 1; k0 < c; k0 += 32) {
        const int k = k0 + (tid >> 3), gl = tid & 7;
        const bool on = k < c;
        T* mk = M + (on ? k : j) * ldm;
        T dot = 0;
        if (on)
          for (int i = j + gl; i < m; i += 8) dot = fma(mj[i], mk[i], dot);
        dot += __shfl_xor_sync(0xffffffffu, dot, 4);
        dot += __shfl_xor_sync(0xffffffffu, dot, 2);
        dot += __shfl_xor_sync(0xffffffffu, dot, 1);
        if (on) {
          const T f = beta * dot;
          for (int i = j + gl; i < m; i += 8) mk[i] = fma(-f, mj[i], mk[i]);
        }
      }
    }
    __syncthreads();
    if (tid == 0) mj[j] = sh_alpha;
    __syncthreads();
  }
  T* Ro = R + (int64_t)tk.out_slot * c * c;
  for (int idx = tid; idx < c * c; idx += 256) {
    const int rr = idx / c, col = idx % c;
    Ro[idx] = (rr <= col && rr < steps) ? M[col * ldm + rr] : (T)0;
  }
}

// Merge of two c x c upper triangular factors: R = qr([R1; R2]).  The j-th
// Householder vector touches row j of R1 and rows 0..j of R2 only, so both
// triangles stay packed (column j holds rows 0..j at offset j (j + 1) / 2).
template <typename T>
__global__ __launch_bounds__(256) void k_tsqr_merge(const TsqrTask* __restrict__ tasks, int c,
                                                    T* __restrict__ R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int pk = c * (c + 1) / 2;
  T* A = reinterpret_cast<T*>(smem_raw);  // R1, packed upper
  T* B = A + pk;                          // R2, packed upper
  __shared__ double red[8];
  __shared__ T sh_alpha, sh_beta, sh_v0;
  const TsqrTask tk = tasks[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* R1 = R + (int64_t)tk.slot[0] * c * c;
  const T* R2 = R + (int64_t)tk.slot[1] * c * c;
  for (int idx = tid; idx < c * c; idx += 256) {
    const int rr = idx / c, col = idx % c;
    if (rr <= col) {
      A[col * (col + 1) / 2 + rr] = R1[idx];
      B[col * (col + 1) / 2 + rr] = R2[idx];
    }
  }
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    const T* bj = B + j * (j + 1) / 2;  // rows 0..j of column j of R2
    T s = 0;
    for (int i = tid; i <= j; i += 256) s = fma(bj[i], bj[i], s);
    s = warp_sum(s);
    if (lane == 0) red[warp] = (double)s;
    __syncthreads();
    if (tid == 0) {
      double tail = 0.0;
      for (int w = 0; w < 8; ++w) tail += red[w];
      const double x0 = (double)A[j * (j + 1) / 2 + j];
      const double nrm = sqrt(x0 * x0 + tail);
      const double alpha = (x0 > 0.0) ? -nrm : nrm;
      const double v0 = x0 - alpha;
      const double vtv = v0 * v0 + tail;
      sh_alpha = (T)alpha;
      sh_v0 = (T)v0;
      sh_beta = (vtv > 0.0) ? (T)(2.0 / vtv) : (T)0;
    }
    __syncthreads();
    const T beta = sh_beta, v0 = sh_v0;
    if (beta != (T)0) {
      // one aligned 8-lane group per trailing column, 32 columns per round
      for (int k0 = j + 1; k0 < c; k0 += 32) {
        const int k = k0 + (tid >> 3), gl = tid & 7;
        const bool on = k < c;
        const int kk = on ? k : j;
        T* ak = A + kk * (kk + 1) / 2;
        T* bk = B + kk * (kk + 1) / 2;
        T dot = 0;
        if (on)
          for (int i = gl; i <= j; i += 8) dot = fma(bj[i], bk[i], dot);
        dot += __shfl_xor_sync(0xffffffffu, dot, 4);
        dot += __shfl_xor_sync(0xffffffffu, dot, 2);
        dot += __shfl_xor_sync(0xffffffffu, dot, 1);
        if (on) {
          const T f = beta * (dot + v0 * ak[j]);
          for (int i = gl; i <= j; i += 8) bk[i] = fma(-f, bj[i], bk[i]);
          if (gl == 0) ak[j] = fma(-f, v0, ak[j]);
        }
      }
    }
    __syncthreads();
    if (tid == 0 && beta != (T)0) A[j * (j + 1) / 2 + j] = sh_alpha;
    __syncthreads();
  }
  T* Ro = R + (int64_t)tk.out_slot * c * c;
  for (int idx = tid; idx < c * c; idx += 256) {
    const int rr = idx / c, col = idx % c;
    Ro[idx] = (rr <= col) ? A[col * (col + 1) / 2 + rr] : (T)0;
  }
}

// One-sided Jacobi SVD of R (c x c) with the rotations accumulated into W;
// round-robin pairing, one warp per pair.  Used in FP32, where it keeps the
// right singular vectors orthonormal to working precision.
template <typename T>
__global__ __launch_bounds__(512) void k_jacobi_acc(const int32_t* __restrict__ node_slot,
                                                const T* __restrict__ R, int c,
                                                T* __restrict__ W, T* __restrict__ sigma) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Am = reinterpret_cast<T*>(smem_raw);  // column j at Am + j * c
  T* Vm = Am + c * c;
  __shared__ int rotated, large;
  __shared__ double sv[128];
  __shared__ int order[128];
  const int node = blockIdx.x;
  const T* Rs = R + (int64_t)node_slot[node] * c * c;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (int idx = tid; idx < c * c; idx += blockDim.x) {
    const int rr = idx / c, col = idx % c;
    Am[col * c + rr] = Rs[idx];
    Vm[col * c + rr] = (rr == col) ? (T)1 : (T)0;
  }
  __syncthreads();
  const int cp = (c + 1) & ~1;  // even number of slots; slot c (odd c) is a bye
  // a pair is rotated while its correlation exceeds the rounding level of the
  // length-c dot products that measure it
  const T tol = (T)(Eps<T>::v * sqrt((double)c));
  const T big2 = (T)(Eps<T>::v * sqrt((double)c));  // (sqrt(tol))^2
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) { rotated = 0; large = 0; }
    __syncthreads();
    for (int step = 0; step < cp - 1; ++step) {
      for (int pi = warp; pi < cp / 2; pi += nwarps) {
        // circle method: slot 0 fixed, the others rotate
        const int a = pi, b = cp - 1 - pi;
        const int p = (a == 0) ? 0 : ((a - 1 + step) % (cp - 1)) + 1;
        const int q = ((b - 1 + step) % (cp - 1)) + 1;
        if (p >= c || q >= c) continue;
        T* ap = Am + p * c;
        T* aq = Am + q * c;
        T alT = 0, beT = 0, gaT = 0;
        for (int i = lane; i < c; i += 32) {
          const T x = ap[i], y = aq[i];
          alT = fma(x, x, alT); beT = fma(y, y, beT); gaT = fma(x, y, gaT);
        }
        const T al = warp_sum(alT), be = warp_sum(beT), ga = warp_sum(gaT);
        // a sweep whose largest correlation stays below sqrt(tol) leaves every
        // pair below tol (quadratic convergence): no confirming sweep needed
        if (lane == 0 && al > (T)0 && be > (T)0 && (ga / al) * (ga / be) > big2) large = 1;
        if (ga != (T)0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          const T zeta = (be - al) / ((T)2 * ga);
          const T t = (zeta >= (T)0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
          const T tc = (T)1 / sqrt((T)1 + t * t), ts = tc * t;
          for (int i = lane; i < c; i += 32) {
            const T x = ap[i], y = aq[i];
            ap[i] = tc * x - ts * y;
            aq[i] = ts * x + tc * y;
          }
          T* vp = Vm + p * c;
          T* vq = Vm + q * c;
          for (int i = lane; i < c; i += 32) {
            const T x = vp[i], y = vq[i];
            vp[i] = tc * x - ts * y;
            vq[i] = ts * x + tc * y;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = rotated && large;
    __syncthreads();
    if (!any) break;
  }
  for (int j = warp; j < c; j += nwarps) {
    T s = 0;
    for (int i = lane; i < c; i += 32) s = fma(Am[j * c + i], Am[j * c + i], s);
    s = warp_sum(s);
    // a non-finite column sorts last (the samples' NaN/Inf flag reports it), so
    // that the ranks below always form a permutation
    if (lane == 0) sv[j] = isfinite((double)s) ? sqrt((double)s) : -1.0;
  }
  __syncthreads();
  for (int j = tid; j < c; j += blockDim.x) {
    int rk = 0;
    for (int i = 0; i < c; ++i) rk += (sv[i] > sv[j]) || (sv[i] == sv[j] && i < j);
    order[rk] = j;
  }
  __syncthreads();
  // sign convention of the singular triplets: the largest-magnitude entry of
  // each right singular vector is positive (the first such entry on ties)
  __shared__ signed char sgn[128];
  for (int j = warp; j < c; j += nwarps) {
    const T* v = Vm + order[j] * c;
    double best = -1.0;
    int bi = c;
    for (int i = lane; i < c; i += 32) {
      const double a = fabs((double)v[i]);
      if (a > best) { best = a; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) sgn[j] = (bi < c && v[bi] < (T)0) ? -1 : 1;
  }
  __syncthreads();
  T* Wn = W + (int64_t)node * c * c;
  for (int idx = tid; idx < c * c; idx += blockDim.x) {
    const int rr = idx % c, col = idx / c;
    Wn[idx] = sgn[col] < 0 ? -Vm[order[col] * c + rr] : Vm[order[col] * c + rr];
  }
  for (int j = tid; j < c; j += blockDim.x) sigma[(int64_t)node * c + j] = (T)sv[order[j]];
}

// FP64 SVD of R (c x c, c <= 128) with the bulk of the Jacobi work in FP32:
//   A. column-pivoted Householder QR R P = Q2 R2 in FP64; X = R2^T (graded
//      columns) is parked in the node's W slot in global memory;
//   B. one-sided Jacobi on float(X) with the rotations accumulated into V32
//      (FP32 arithmetic, FP32 convergence threshold);
//   C. Q = CGS2 orthonormalization of V32 in FP64 (orthogonal to FP64
//      rounding; it differs from the exact V only by the FP32 error of B);
//   D. X1 = X Q in FP64: same left singular vectors as X, columns orthogonal
//      to FP32 precision;
//   E. one-sided Jacobi on X1 in FP64 until the FP64 threshold holds (one or
//      two sweeps from an FP32-orthogonal start);
//   F. sigma_j = |X1_j|, right singular vectors of R: W = P U_x, U_x = the
//      normalized columns; sorted descending, sign convention as in k_jacobi_acc.
__global__ __launch_bounds__(512) void k_jacobi_mp(const int32_t* __restrict__ node_slot,
                                                   const double* __restrict__ R, int c,
                                                   double* __restrict__ W,
                                                   double* __restrict__ sigma) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* M = reinterpret_cast<double*>(smem_raw);  // phase A: c x c, column-major
  float* V32 = reinterpret_cast<float*>(smem_raw);  // phases B-C: c x c
  const size_t off_q = (((size_t)c * c * sizeof(float)) + 15) & ~(size_t)15;
  float* X32 = reinterpret_cast<float*>(smem_raw + off_q);    // phase B
  double* Q = reinterpret_cast<double*>(smem_raw + off_q);    // phases C-F (X1 after D)
  __shared__ int rotated, large;
  __shared__ double sv[128];
  __shared__ double cn[128];
  __shared__ double hb[128];
  __shared__ int perm[128];
  __shared__ int order[128];
  __shared__ signed char sgn[128];
  __shared__ double red_v[16];
  __shared__ int red_i[16];
  __shared__ double sh_alpha, sh_beta;
  __shared__ double psum[4][128];  // C: partial projections
  const int node = blockIdx.x;
  const double* Rs = R + (int64_t)node_slot[node] * c * c;
  double* Wn = W + (int64_t)node * c * c;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int nthr = blockDim.x;
  const int pg = tid >> 3, gl = tid & 7;  // sweeps: pair slot (8 lanes each), lane in it
  // ---------------------------------------------------------------- A
  for (int idx = tid; idx < c * c; idx += nthr) {
    const int rr = idx / c, col = idx % c;
    M[col * c + rr] = Rs[idx];
  }
  for (int j = tid; j < c; j += nthr) perm[j] = j;
  __syncthreads();
  // squared norms of the trailing columns: computed once, downdated after every
  // step (cn[k] -= M(j, k)^2) and recomputed where the downdate has cancelled
  // below sqrt(eps) of the last computed value (hb[] keeps that value)
  for (int k = warp; k < c; k += nwarps) {
    const double* mk = M + k * c;
    double s = 0;
    for (int i = lane; i < c; i += 32) s = fma(mk[i], mk[i], s);
    s = warp_sum(s);
    if (lane == 0) { cn[k] = s; hb[k] = s; }
  }
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    for (int k = j + warp; k < c; k += nwarps) {
      if (!(cn[k] > 1.4901161193847656e-08 * hb[k])) {
        const double* mk = M + k * c;
        double s = 0;
        for (int i = j + lane; i < c; i += 32) s = fma(mk[i], mk[i], s);
        s = warp_sum(s);
        if (lane == 0) { cn[k] = s; hb[k] = s; }
      }
    }
    __syncthreads();
    if (warp == 0) {
      double best = -1.0;
      int bi = c;
      for (int k = j + lane; k < c; k += 32)
        if (cn[k] > best) { best = cn[k]; bi = k; }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { red_i[0] = bi; red_v[0] = best; }
    }
    __syncthreads();
    const int p = red_i[0];
    if (p != j && p < c) {
      for (int i = tid; i < c; i += nthr) {
        const double t = M[j * c + i];
        M[j * c + i] = M[p * c + i];
        M[p * c + i] = t;
      }
      if (tid == 0) {
        const int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
        double u = cn[j]; cn[j] = cn[p]; cn[p] = u;
        u = hb[j]; hb[j] = hb[p]; hb[p] = u;
      }
    }
    __syncthreads();
    double* mj = M + j * c;
    if (warp == 0) {  // the reflector needs the pivot column's exact norm
      double s = 0;
      for (int i = j + lane; i < c; i += 32) s = fma(mj[i], mj[i], s);
      s = warp_sum(s);
      if (lane == 0) red_v[0] = s;
    }
    __syncthreads();
    if (tid == 0) {
      const double tot = red_v[0] > 0.0 ? red_v[0] : 0.0;
      const double x0 = mj[j];
      const double nrm = sqrt(tot);
      const double alpha = (x0 > 0.0) ? -nrm : nrm;
      const double v0 = x0 - alpha;
      const double vtv = tot - x0 * x0 + v0 * v0;
      sh_alpha = alpha;
      sh_beta = (vtv > 0.0) ? 2.0 / vtv : 0.0;
      mj[j] = v0;
    }
    __syncthreads();
    const double beta = sh_beta;
    if (beta != 0.0) {
      for (int k0 = j + 1; k0 < c; k0 += 64) {  // one 8-lane group per trailing column
        const int k = k0 + pg;
        const bool on = k < c;
        double* mk = M + (on ? k : j) * c;
        double dot = 0;
        if (on)
          for (int i = j + gl; i < c; i += 8) dot = fma(mj[i], mk[i], dot);
        dot += __shfl_xor_sync(0xffffffffu, dot, 4);
        dot += __shfl_xor_sync(0xffffffffu, dot, 2);
        dot += __shfl_xor_sync(0xffffffffu, dot, 1);
        if (on) {
          const double f = beta * dot;
          for (int i = j + gl; i < c; i += 8) mk[i] = fma(-f, mj[i], mk[i]);
        }
      }
    }
    __syncthreads();
    if (tid == 0 && beta != 0.0) mj[j] = sh_alpha;
    for (int k = j + 1 + tid; k < c; k += nthr) cn[k] -= M[k * c + j] * M[k * c + j];
    __syncthreads();
  }
  // X = R2^T, column-major, parked in the W slot
  for (int idx = tid; idx < c * c; idx += nthr) {
    const int col = idx / c, row = idx % c;  // X(row, col) = R2(col, row), zero above
    Wn[idx] = (row >= col) ? M[row * c + col] : 0.0;
  }
  __syncthreads();
  // ---------------------------------------------------------------- B
  for (int idx = tid; idx < c * c; idx += nthr) {
    X32[idx] = (float)Wn[idx];
    V32[idx] = (idx / c == idx % c) ? 1.f : 0.f;
  }
  __syncthreads();
  const int cp = (c + 1) & ~1;
  // squared column norms of X32, updated by each rotation (hb[] as FP32 storage)
  float* cn32 = reinterpret_cast<float*>(hb);
  for (int j = warp; j < c; j += nwarps) {
    float s2 = 0.f;
    for (int i = lane; i < c; i += 32) s2 = fmaf(X32[j * c + i], X32[j * c + i], s2);
    s2 = warp_sum(s2);
    if (lane == 0) cn32[j] = s2;
  }
  __syncthreads();
  {
    const float tol = (float)(Eps<float>::v * sqrt((double)c));
    const float big2 = tol;  // (sqrt(tol))^2
    for (int sweep = 0; sweep < 40; ++sweep) {
      if (tid == 0) { rotated = 0; large = 0; }
      __syncthreads();
      for (int step = 0; step < cp - 1; ++step) {
        // all pairs of the step at once, one aligned 8-lane group per pair
        int p = c, q = c;
        if (pg < cp / 2) {
          const int a = pg, b = cp - 1 - pg;
          p = (a == 0) ? 0 : ((a - 1 + step) % (cp - 1)) + 1;
          q = ((b - 1 + step) % (cp - 1)) + 1;
        }
        const bool valid = p < c && q < c;
        float* ap = X32 + (valid ? p : 0) * c;
        float* aq = X32 + (valid ? q : 0) * c;
        float ga = 0;
        if (valid)
          for (int i = gl; i < c; i += 8) ga = fmaf(ap[i], aq[i], ga);
        ga += __shfl_xor_sync(0xffffffffu, ga, 4);
        ga += __shfl_xor_sync(0xffffffffu, ga, 2);
        ga += __shfl_xor_sync(0xffffffffu, ga, 1);
        if (valid) {
          const float al = cn32[p], be = cn32[q];
          if (gl == 0 && al > 0.f && be > 0.f && (ga / al) * (ga / be) > big2) large = 1;
          if (ga != 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be)) {
            const float zeta = (be - al) / (2.f * ga);
            const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
            const float tc = 1.f / sqrtf(1.f + t * t), ts = tc * t;
            for (int i = gl; i < c; i += 8) {
              const float x = ap[i], y = aq[i];
              ap[i] = tc * x - ts * y;
              aq[i] = ts * x + tc * y;
            }
            float* vp = V32 + p * c;
            float* vq = V32 + q * c;
            for (int i = gl; i < c; i += 8) {
              const float x = vp[i], y = vq[i];
              vp[i] = tc * x - ts * y;
              vq[i] = ts * x + tc * y;
            }
            if (gl == 0) {
              const float cs2 = 2.f * tc * ts, c2 = tc * tc, s2 = ts * ts;
              cn32[p] = fmaxf(fmaf(c2, al, fmaf(-cs2, ga, s2 * be)), 0.f);
              cn32[q] = fmaxf(fmaf(s2, al, fmaf(cs2, ga, c2 * be)), 0.f);
              rotated = 1;
            }
          }
        }
        __syncthreads();
      }
      const int any = rotated && large;
      __syncthreads();
      if (!any) break;
    }
  }
  // ---------------------------------------------------------------- C
  // (X32 is dead; Q overlays it)
  for (int j = 0; j < c; ++j) {
    double* qj = Q + j * c;
    for (int i = tid; i < c; i += nthr) qj[i] = (double)V32[j * c + i];
    __syncthreads();
    // one classical Gram-Schmidt pass: V32 is orthogonal to FP32 precision, and
    // CGS loses orthogonality in proportion to cond(V32)^2 ~ 1
    {
      for (int i0 = 0; i0 < j; i0 += 64) {  // one 8-lane group per earlier column
        const int i = i0 + pg;
        const bool on = i < j;
        const double* qi = Q + (on ? i : 0) * c;
        double s = 0;
        if (on)
          for (int e = gl; e < c; e += 8) s = fma(qi[e], qj[e], s);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (on && gl == 0) hb[i] = s;
      }
      __syncthreads();
      {  // q_j -= sum_i hb[i] Q_i in four partial sums over quarters of i
        const int e = tid & 127, part = tid >> 7;
        const int i0 = (j * part) >> 2, i1 = (j * (part + 1)) >> 2;
        double s = 0;
        if (e < c)
          for (int i = i0; i < i1; ++i) s = fma(hb[i], Q[i * c + e], s);
        psum[part][e] = s;
      }
      __syncthreads();
      for (int e = tid; e < c; e += nthr)
        qj[e] -= (psum[0][e] + psum[1][e]) + (psum[2][e] + psum[3][e]);
      __syncthreads();
    }
    if (warp == 0) {
      double s = 0;
      for (int e = lane; e < c; e += 32) s = fma(qj[e], qj[e], s);
      s = warp_sum(s);
      if (lane == 0) hb[0] = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
    }
    __syncthreads();
    const double inv = hb[0];
    for (int e = tid; e < c; e += nthr) qj[e] *= inv;
    __syncthreads();
  }
  // ---------------------------------------------------------------- D
  for (int j = warp; j < c; j += nwarps) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const double* qj = Q + j * c;
    for (int k = 0; k < c; ++k) {
      const double qk = qj[k];
      const double* xk = Wn + (int64_t)k * c;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int row = lane + 32 * rr;
        if (row < c) acc[rr] = fma(xk[row], qk, acc[rr]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int row = lane + 32 * rr;
      if (row < c) Q[j * c + row] = acc[rr];
    }
  }
  __syncthreads();
  // ---------------------------------------------------------------- E
  // The squared column norms live in cn[] and each rotation updates them from
  // (al, be, ga), so a pair costs one dot product.  Starting from X1, whose
  // columns are orthogonal to FP32 precision, nearly every angle is tiny: then
  // t = tan(theta) = u - u^3 + ..., u = ga / (be - al), from an approximate FP64
  // reciprocal refined by one Newton step (so that the confirming sweep finds
  // nothing left to rotate), and
  // cos = 1 - t^2/2 + 3t^4/8, sin = t cos, which is orthogonal to FP64
  // rounding for |t| < 2^-10 (the dropped terms are below t^6).  Larger angles
  // take the exact formulas.  The final norms are recomputed in F.
  for (int j = warp; j < c; j += nwarps) {
    double s2 = 0;
    for (int i = lane; i < c; i += 32) s2 = fma(Q[j * c + i], Q[j * c + i], s2);
    s2 = warp_sum(s2);
    if (lane == 0) cn[j] = s2;
  }
  __syncthreads();
  {
    const double tol = Eps<double>::v * sqrt((double)c);
    const double tol2 = tol * tol, big2 = tol;  // squared thresholds
    for (int sweep = 0; sweep < 12; ++sweep) {
      if (tid == 0) { rotated = 0; large = 0; }
      __syncthreads();
      for (int step = 0; step < cp - 1; ++step) {
        int p = c, q = c;  // one aligned 8-lane group per pair, as in B
        if (pg < cp / 2) {
          const int a = pg, b = cp - 1 - pg;
          p = (a == 0) ? 0 : ((a - 1 + step) % (cp - 1)) + 1;
          q = ((b - 1 + step) % (cp - 1)) + 1;
        }
        const bool valid = p < c && q < c;
        double* ap = Q + (valid ? p : 0) * c;
        double* aq = Q + (valid ? q : 0) * c;
        double ga = 0;
        if (valid)
          for (int i = gl; i < c; i += 8) ga = fma(ap[i], aq[i], ga);
        ga += __shfl_xor_sync(0xffffffffu, ga, 4);
        ga += __shfl_xor_sync(0xffffffffu, ga, 2);
        ga += __shfl_xor_sync(0xffffffffu, ga, 1);
        if (valid) {
          const double al = cn[p], be = cn[q];
          const double g2 = ga * ga, ab = al * be;
          if (gl == 0 && g2 > big2 * ab) large = 1;
          if (ga != 0.0 && g2 > tol2 * ab) {
            const double d = be - al;
            double tc, ts;
            if (fabs(ga) < 0.00048828125 * fabs(d) && fabs(d) > 1e-290) {  // |t| < 2^-11
              double r;
              asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
              r = fma(r, fma(-d, r, 1.0), r);      // one Newton step: FP64-accurate
              const double u = ga * r;             // 1 / (2 zeta)
              const double t = fma(-u * u, u, u);  // tan(theta) = u - u^3 + ...
              const double t2 = t * t;
              tc = fma(t2, fma(t2, 0.375, -0.5), 1.0);
              ts = tc * t;
            } else {
              const double zeta = d / (2.0 * ga);
              const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
              tc = 1.0 / sqrt(1.0 + t * t);
              ts = tc * t;
            }
            for (int i = gl; i < c; i += 8) {
              const double x = ap[i], y = aq[i];
              ap[i] = tc * x - ts * y;
              aq[i] = ts * x + tc * y;
            }
            if (gl == 0) {
              // norms after the rotation (whatever the angle's accuracy)
              const double cs2 = 2.0 * tc * ts, c2 = tc * tc, s2 = ts * ts;
              cn[p] = fma(c2, al, fma(-cs2, ga, s2 * be));
              cn[q] = fma(s2, al, fma(cs2, ga, c2 * be));
              rotated = 1;
            }
          }
        }
        __syncthreads();
      }
      const int any = rotated && large;
      __syncthreads();
      if (!any) break;
    }
  }
  // ---------------------------------------------------------------- F
  for (int j = warp; j < c; j += nwarps) {
    double s = 0;
    for (int i = lane; i < c; i += 32) s = fma(Q[j * c + i], Q[j * c + i], s);
    s = warp_sum(s);
    if (lane == 0) sv[j] = isfinite(s) ? sqrt(s) : -1.0;
  }
  __syncthreads();
  for (int j = tid; j < c; j += nthr) {
    int rk = 0;
    for (int i = 0; i < c; ++i) rk += (sv[i] > sv[j]) || (sv[i] == sv[j] && i < j);
    order[rk] = j;
  }
  __syncthreads();
  for (int j = warp; j < c; j += nwarps) {
    const double* x = Q + order[j] * c;
    double best = -1.0, bv = 0.0;
    int bi = c;
    for (int i = lane; i < c; i += 32) {
      const double a = fabs(x[i]);
      const int row = perm[i];
      if (a > best || (a == best && row < bi)) { best = a; bi = row; bv = x[i]; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; bv = ov; }
    }
    if (lane == 0) sgn[j] = (bv < 0.0) ? -1 : 1;
  }
  __syncthreads();
  for (int idx = tid; idx < c * c; idx += nthr) {
    const int i = idx % c, col = idx / c;
    const int j = order[col];
    const double s = sv[j];
    const double u = (s > 0.0) ? Q[j * c + i] / s : 0.0;
    Wn[perm[i] + col * c] = sgn[col] < 0 ? -u : u;
  }
  for (int j = tid; j < c; j += nthr) sigma[(int64_t)node * c + j] = sv[order[j]] > 0.0 ? sv[order[j]] : 0.0;
}

template <typename T>
__global__ void k_truncate(int nnodes, const T* __restrict__ W, const T* __restrict__ sigma,
                           int c, int kcap, int mode, int kfix, double tol_scaled,
                           double* __restrict__ eps_abs, int set_eps, double floor_rel,
                           int32_t* __restrict__ rank, T* __restrict__ T1,
                           int32_t* __restrict__ saturated) {
  __shared__ int sk;
  const int node = blockIdx.x;
  const T* sg = sigma + (int64_t)node * c;
  if (threadIdx.x == 0) {
    const double s1 = (double)sg[0];
    double thr = floor_rel * s1;
    if (mode == 1) {
      double eps;
      if (set_eps) {
        double nu = 0.0;
        for (int i = 0; i < nnodes; ++i) nu = fmax(nu, (double)sigma[(int64_t)i * c]);
        eps = tol_scaled * nu;
        if (node == 0) *eps_abs = eps;
      } else {
        eps = *eps_abs;
      }
      thr = fmax(thr, eps);
    }
    int k = 0;
    const int lim = c < kcap ? c : kcap;
    while (k < lim && (double)sg[k] > thr) ++k;
    if (mode == 2) {
      int kk = kfix < lim ? kfix : lim;
      while (kk > 0 && !((double)sg[kk - 1] > 0.0)) --kk;
      k = kk;
    }
    if (mode == 1 && k == lim && lim < c && (double)sg[lim] > thr) atomicAdd(saturated, 1);
    if (mode == 1 && k == lim && lim == c) atomicAdd(saturated, 1);
    if (k < 1 && (double)sg[0] > 0.0) k = 1;
    rank[node] = k;
    sk = k;
  }
  __syncthreads();
  const int k = sk;
  const T* Wn = W + (int64_t)node * c * c;
  T* Tn = T1 + (int64_t)node * c * kcap;
  for (int idx = threadIdx.x; idx < c * kcap; idx += blockDim.x) {
    const int rr = idx % c, col = idx / c;
    Tn[idx] = (col < k) ? (T)((double)Wn[rr + col * c] / (double)sg[col]) : (T)0;
  }
}

// CholQR: G (kcap x kcap) = Q1^T Q1 -> R2 = chol(G) (dead pivots dropped),
// T2 = R2^{-1}; optionally M = W_k S_k R2^T (c x kcap).
template <typename T>
__global__ __launch_bounds__(256) void k_cholqr(const T* __restrict__ G, int kcap,
                                                const int32_t* __restrict__ rank,
                                                T* __restrict__ T2, const T* __restrict__ W,
                                                const T* __restrict__ sigma, int c,
                                                T* __restrict__ M, int want_m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Rm = reinterpret_cast<T*>(smem_raw);  // kcap x kcap, row-major upper
  T* Ti = Rm + kcap * kcap;                 // kcap x kcap inverse, row-major
  __shared__ int dead[128];
  const int node = blockIdx.x;
  const int k = rank[node];
  const T* Gn = G + (int64_t)node * kcap * kcap;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kcap * kcap; idx += blockDim.x) {
    const int i = idx / kcap, j = idx % kcap;
    Rm[idx] = (i < k && j < k) ? Gn[i + j * kcap] : (T)0;
    Ti[idx] = 0;
  }
  for (int j = tid; j < kcap; j += blockDim.x) dead[j] = (j >= k);
  __syncthreads();
  double dmax = 0.0;
  for (int j = 0; j < k; ++j) dmax = fmax(dmax, (double)Rm[j * kcap + j]);
  // right-looking Cholesky, upper factor in Rm; a pivot below 64 eps max(diag)
  // marks a dependent column, which is dropped
  __shared__ double piv;
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      const double d = (double)Rm[j * kcap + j];
      if (dead[j] || !(d > 64.0 * Eps<T>::v * dmax)) {
        dead[j] = 1;
        piv = 0.0;
      } else {
        piv = sqrt(d);
      }
    }
    __syncthreads();
    const T pj = (T)piv;
    if (pj == (T)0) {
      for (int l = j + tid; l < kcap; l += blockDim.x) Rm[j * kcap + l] = (l == j) ? (T)1 : (T)0;
      __syncthreads();
      continue;
    }
    for (int l = j + tid; l < k; l += blockDim.x) Rm[j * kcap + l] /= pj;  // R(j,j) = sqrt(d)
    __syncthreads();
    // trailing update of the upper triangle: G(a,b) -= R(j,a) R(j,b), a <= b
    const int rem = k - j - 1;
    for (int idx = tid; idx < rem * rem; idx += blockDim.x) {
      const int a = j + 1 + idx / rem, b = j + 1 + idx % rem;
      if (a <= b) Rm[a * kcap + b] = fma(-Rm[j * kcap + a], Rm[j * kcap + b], Rm[a * kcap + b]);
    }
    __syncthreads();
  }
  // inverse of the upper-triangular R2, one column per thread; dead columns -> 0
  for (int l = tid; l < kcap; l += blockDim.x) {
    if (l >= k || dead[l]) continue;
    Ti[l * kcap + l] = (T)1 / Rm[l * kcap + l];
    for (int i = l - 1; i >= 0; --i) {
      if (dead[i]) continue;
      T s = 0;
      for (int mm = i + 1; mm <= l; ++mm) s = fma(Rm[i * kcap + mm], Ti[mm * kcap + l], s);
      Ti[i * kcap + l] = -s / Rm[i * kcap + i];
    }
  }
  __syncthreads();
  T* T2n = T2 + (int64_t)node * kcap * kcap;
  for (int idx = tid; idx < kcap * kcap; idx += blockDim.x) {
    const int i = idx % kcap, j = idx / kcap;  // column-major output
    T2n[idx] = Ti[i * kcap + j];
  }
  if (want_m) {
    // M(row, col) = sum_{m >= col} W(row, m) s_m R2(col, m), live columns only
    const T* Wn = W + (int64_t)node * c * c;
    const T* sg = sigma + (int64_t)node * c;
    T* Mn = M + (int64_t)node * c * kcap;
    for (int idx = tid; idx < c * kcap; idx += blockDim.x) {
      const int row = idx % c, col = idx / c;
      T s = 0;
      if (col < k && !dead[col])
        for (int mm = col; mm < k; ++mm)
          if (!dead[mm]) s = fma(Wn[row + mm * c] * sg[mm], Rm[col * kcap + mm], s);
      Mn[idx] = s;
    }
  }
}

}  // namespace

template <typename T>
void launch_tsqr(const TsqrTask* tasks, int ntasks, int merge, const T* P, int64_t ldp, int c,
                 T* R, cudaStream_t st) {
  count_launches(1);
  if (!merge) {
    // columns 136 entries apart: the four 8-lane groups of a warp then fall on
    // two bank halves (the two wavefronts a 256-byte access takes anyway)
    const int ldm = kTsqrRows + 8;
    const size_t smem = (size_t)ldm * c * sizeof(T);
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_tsqr<T>, done);
    k_tsqr<T><<<ntasks, 256, smem, st>>>(tasks, P, ldp, c, R, ldm);
  } else {
    const size_t smem = (size_t)c * (c + 1) * sizeof(T);
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_tsqr_merge<T>, done);
    k_tsqr_merge<T><<<ntasks, 256, smem, st>>>(tasks, c, R);
  }
}

template <typename T>
void launch_jacobi(const int32_t* node_slot, int nnodes, const T* R, int c, T* W, T* sigma,
                   cudaStream_t st) {
  count_launches(1);
  int threads = ((c / 2 + 31) / 32) * 32 * 32;
  if (threads > 512) threads = 512;
  if (threads < 64) threads = 64;
  if (sizeof(T) == 4) {
    const size_t smem = (size_t)2 * c * c * sizeof(T);
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_jacobi_acc<T>, done);
    k_jacobi_acc<T><<<nnodes, threads, smem, st>>>(node_slot, R, c, W, sigma);
  } else {
    const size_t off_q = (((size_t)c * c * sizeof(float)) + 15) & ~(size_t)15;
    const size_t smem = std::max((size_t)c * c * sizeof(double), off_q + (size_t)c * c * sizeof(double));
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_jacobi_mp, done);
    // the sweeps give each of the (c + 1) / 2 <= 64 pairs of a step 8 lanes
    k_jacobi_mp<<<nnodes, 512, smem, st>>>(node_slot, (const double*)R, c, (double*)W,
                                               (double*)sigma);
  }
}

template <typename T>
void launch_truncate(int nnodes, const T* W, const T* sigma, int c, int kcap, int mode, int kfix,
                     double tol_scaled, double* eps_abs, int set_eps, double floor_rel,
                     int32_t* rank, T* T1, int32_t* saturated, cudaStream_t st) {
  count_launches(1);
  k_truncate<T><<<nnodes, 128, 0, st>>>(nnodes, W, sigma, c, kcap, mode, kfix, tol_scaled,
                                        eps_abs, set_eps, floor_rel, rank, T1, saturated);
}

template <typename T>
void launch_cholqr(int nnodes, const T* G, int kcap, const int32_t* rank, T* T2, const T* W,
                   const T* sigma, int c, T* M, int want_m, cudaStream_t st) {
  count_launches(1);
  const size_t smem = (size_t)2 * kcap * kcap * sizeof(T);
  static std::atomic<uint32_t> done{0};
  raise_smem_limit((const void*)k_cholqr<T>, done);
  k_cholqr<T><<<nnodes, 256, smem, st>>>(G, kcap, rank, T2, W, sigma, c, M, want_m);
}

#define HM_INST(T)                                                                           \
  template void launch_tsqr<T>(const TsqrTask*, int, int, const T*, int64_t, int, T*,        \
                               cudaStream_t);                                                \
  template void launch_jacobi<T>(const int32_t*, int, const T*, int, T*, T*, cudaStream_t);  \
  template void launch_truncate<T>(int, const T*, const T*, int, int, int, int, double,      \
                                   double*, int, double, int32_t*, T*, int32_t*,             \
                                   cudaStream_t);                                            \
  template void launch_cholqr<T>(int, const T*, int, const int32_t*, T*, const T*, const T*, \
                                 int, T*, int, cudaStream_t);
HM_INST(float)
HM_INST(double)
#undef HM_INST

}  // namespace hm
