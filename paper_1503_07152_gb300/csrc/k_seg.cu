// Segmented (per tree node) tall-skinny products, the workhorses of the peel
// and of the per-node linear algebra:
//   seg_tn:  out[node] = A(I_node, :)^T B(I_node, :)   (projections V^T x of the
//            HODLR product, Sec. 2.8; Gram matrices; the short-basis products
//            U_alpha^* U_tau(J_alpha,:) of Fig. "A basic scheme for compressing an
//            HBS matrix")
//   seg_nn:  Y(I_node, :) = alpha P(I_node, :) C[node'] + beta Y(I_node, :)
//            (expansions U t, basis updates U <- U \hat U, Q = P T).
// A node's rows are split into chunks; uneven node sizes go into one launch.
// Column offsets can depend on the node's parity (left child / right child), which
// is how the packed test matrices [Omega_2 | Omega_1] are addressed.
#include <atomic>

#include "hm_internal.h"

namespace hm {
namespace {

constexpr int TN_ROWS = 32;   // rows staged per step
constexpr int TN_MAX = 128;   // max ka, kb

// Per-thread tile for a product of ka x kb outputs: 256 threads in a 16 x 16
// grid, thread (ti, tj) owning rows ti + 16 i (i < TI) and columns tj + 16 j
// (j < TJ), so a warp reads 16 consecutive staged columns of B (no bank
// conflicts) and only the 16 TI x 16 TJ outputs that cover ka x kb are computed.
// Which thread owns an output changes nothing in how it is summed.
constexpr int tn_tile(int k) { return k <= 32 ? 2 : (k <= 64 ? 4 : 8); }

// Partial products of one chunk (<= 256 rows).
template <typename T, int TI, int TJ>
__global__ __launch_bounds__(256) void k_seg_tn_partial(
    const Chunk* __restrict__ chunks, const T* __restrict__ A, int64_t lda, int aoff_e,
    int aoff_o, int ka, const T* __restrict__ B, int64_t ldb, int boff_e, int boff_o, int kb,
    double* __restrict__ partial) {
  constexpr int KA = 16 * TI, KB = 16 * TJ, LDA = KA + 1, LDB = KB + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);  // [TN_ROWS][LDA]
  T* Bs = As + TN_ROWS * LDA;              // [TN_ROWS][LDB]
  const Chunk ch = chunks[blockIdx.x];
  const int aoff = (ch.node & 1) ? aoff_o : aoff_e;
  const int boff = (ch.node & 1) ? boff_o : boff_e;
  const int tid = threadIdx.x;
  const int ti = tid >> 4, tj = tid & 15;
  // products summed in T over at most 16 rows, then added into FP64 sums: the
  // projections of the peel are differences of large sums, so a long FP32 sum
  // would cost far more than its unit roundoff
  double acc[TI][TJ];
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int j = 0; j < TJ; ++j) acc[i][j] = 0.0;
  for (int64_t r0 = ch.r0; r0 < ch.r1; r0 += TN_ROWS) {
    const int rows = (int)((ch.r1 - r0) < TN_ROWS ? (ch.r1 - r0) : TN_ROWS);
    for (int idx = tid; idx < TN_ROWS * KA; idx += 256) {
      const int rr = idx % TN_ROWS, c = idx / TN_ROWS;
      As[rr * LDA + c] = (rr < rows && c < ka) ? A[r0 + rr + (int64_t)(aoff + c) * lda] : (T)0;
    }
    for (int idx = tid; idx < TN_ROWS * KB; idx += 256) {
      const int rr = idx % TN_ROWS, c = idx / TN_ROWS;
      Bs[rr * LDB + c] = (rr < rows && c < kb) ? B[r0 + rr + (int64_t)(boff + c) * ldb] : (T)0;
    }
    __syncthreads();
    for (int q0 = 0; q0 < rows; q0 += 16) {
      const int q1 = (q0 + 16 < rows) ? q0 + 16 : rows;
      T tmp[TI][TJ];
#pragma unroll
      for (int i = 0; i < TI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) tmp[i][j] = 0;
      for (int rr = q0; rr < q1; ++rr) {
        T a[TI], b[TJ];
#pragma unroll
        for (int i = 0; i < TI; ++i) a[i] = As[rr * LDA + ti + 16 * i];
#pragma unroll
        for (int j = 0; j < TJ; ++j) b[j] = Bs[rr * LDB + tj + 16 * j];
#pragma unroll
        for (int i = 0; i < TI; ++i)
#pragma unroll
          for (int j = 0; j < TJ; ++j) tmp[i][j] = fma(a[i], b[j], tmp[i][j]);
      }
#pragma unroll
      for (int i = 0; i < TI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) acc[i][j] += (double)tmp[i][j];
    }
    __syncthreads();
  }
  double* out = partial + (int64_t)blockIdx.x * ka * kb;
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int j = 0; j < TJ; ++j) {
      const int ii = ti + 16 * i, jj = tj + 16 * j;
      if (ii < ka && jj < kb) out[ii + jj * ka] = acc[i][j];
    }
}

// The FP64 form of the partial products in double-float arithmetic on the FP32
// pipe (GB300's FP64 pipe runs at a small fraction of the FP32 rate).  Each FP64
// input is cut once, when staged, into x = hi + lo (two floats, 48 significant
// bits); a product a b is formed as hi_a hi_b exactly (TwoProduct by FMA) plus
// the cross terms, and summed per output in a double-float (s_hi, s_lo) through
// TwoSum.  The partial of a chunk (<= 256 rows) is accurate to ~1e-14 relative.
__device__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

template <int TI, int TJ>
__global__ __launch_bounds__(256) void k_seg_tn_partial_df(
    const Chunk* __restrict__ chunks, const double* __restrict__ A, int64_t lda, int aoff_e,
    int aoff_o, int ka, const double* __restrict__ B, int64_t ldb, int boff_e, int boff_o,
    int kb, double* __restrict__ partial) {
  constexpr int KA = 16 * TI, KB = 16 * TJ, LDA = KA + 1, LDB = KB + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ah = reinterpret_cast<float*>(smem_raw);  // [TN_ROWS][LDA] each
  float* Al = Ah + TN_ROWS * LDA;
  float* Bh = Al + TN_ROWS * LDA;                  // [TN_ROWS][LDB] each
  float* Bl = Bh + TN_ROWS * LDB;
  const Chunk ch = chunks[blockIdx.x];
  const int aoff = (ch.node & 1) ? aoff_o : aoff_e;
  const int boff = (ch.node & 1) ? boff_o : boff_e;
  const int tid = threadIdx.x;
  const int ti = tid >> 4, tj = tid & 15;
  float sh[TI][TJ], sl[TI][TJ];
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int j = 0; j < TJ; ++j) { sh[i][j] = 0.f; sl[i][j] = 0.f; }
  for (int64_t r0 = ch.r0; r0 < ch.r1; r0 += TN_ROWS) {
    const int rows = (int)((ch.r1 - r0) < TN_ROWS ? (ch.r1 - r0) : TN_ROWS);
    for (int idx = tid; idx < TN_ROWS * KA; idx += 256) {
      const int rr = idx % TN_ROWS, c = idx / TN_ROWS;
      float h, l;
      split_df((rr < rows && c < ka) ? A[r0 + rr + (int64_t)(aoff + c) * lda] : 0.0, h, l);
      Ah[rr * LDA + c] = h;
      Al[rr * LDA + c] = l;
    }
    for (int idx = tid; idx < TN_ROWS * KB; idx += 256) {
      const int rr = idx % TN_ROWS, c = idx / TN_ROWS;
      float h, l;
      split_df((rr < rows && c < kb) ? B[r0 + rr + (int64_t)(boff + c) * ldb] : 0.0, h, l);
      Bh[rr * LDB + c] = h;
      Bl[rr * LDB + c] = l;
    }
    __syncthreads();
    for (int rr = 0; rr < rows; ++rr) {
      float ah[TI], al[TI], bh[TJ], bl[TJ];
#pragma unroll
      for (int i = 0; i < TI; ++i) {
        ah[i] = Ah[rr * LDA + ti + 16 * i];
        al[i] = Al[rr * LDA + ti + 16 * i];
      }
#pragma unroll
      for (int j = 0; j < TJ; ++j) {
        bh[j] = Bh[rr * LDB + tj + 16 * j];
        bl[j] = Bl[rr * LDB + tj + 16 * j];
      }
#pragma unroll
      for (int i = 0; i < TI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) {
          const float p = ah[i] * bh[j];
          const float e = fmaf(ah[i], bh[j], -p);               // hi hi - p, exact
          const float t = fmaf(ah[i], bl[j], fmaf(al[i], bh[j], e));
          const float s = sh[i][j] + p;                          // TwoSum(sh, p)
          const float z = s - sh[i][j];
          const float err = (sh[i][j] - (s - z)) + (p - z);
          sh[i][j] = s;
          sl[i][j] += err + t;
        }
    }
    __syncthreads();
  }
  double* out = partial + (int64_t)blockIdx.x * ka * kb;
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int j = 0; j < TJ; ++j) {
      const int ii = ti + 16 * i, jj = tj + 16 * j;
      if (ii < ka && jj < kb) out[ii + jj * ka] = (double)sh[i][j] + (double)sl[i][j];
    }
}

// out[node] = sum of the node's chunk partials, in chunk order (deterministic).
template <typename T>
__global__ void k_seg_tn_reduce(const double* __restrict__ partial,
                                const int32_t* __restrict__ chunk_begin, int ka, int kb,
                                T* __restrict__ out) {
  const int node = blockIdx.y;
  const int c0 = chunk_begin[node], c1 = chunk_begin[node + 1];
  const int m = ka * kb;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = c0; c < c1; ++c) s += partial[(int64_t)c * m + e];
    out[(int64_t)node * m + e] = (T)s;
  }
}

constexpr int NN_ROWS = 64;
constexpr int NN_MAX = 128;

// One chunk of <= 64 rows.  Warp w owns output columns [16w, 16w + 16); lane
// owns rows lane and lane + 32.  P is staged before any write (in-place safe).
template <typename T>
__global__ __launch_bounds__(256) void k_seg_nn(
    const Chunk* __restrict__ chunks, int node0, const T* P, int64_t ldp, int poff_e,
    int poff_o, int kin, const T* __restrict__ C, int64_t cstride, int cld, int cflip, T* Y,
    int64_t ldy, int yoff_e, int yoff_o, int kout, T alpha, T beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ps = reinterpret_cast<T*>(smem_raw);   // [NN_MAX][NN_ROWS]
  T* Cs = Ps + NN_MAX * NN_ROWS;             // [NN_MAX][NN_MAX]
  const Chunk ch = chunks[blockIdx.x];
  const int rows = (int)(ch.r1 - ch.r0);
  const int poff = (ch.node & 1) ? poff_o : poff_e;
  const int yoff = (ch.node & 1) ? yoff_o : yoff_e;
  const T* Cn = C + (int64_t)((ch.node ^ cflip) - node0) * cstride;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kin * NN_ROWS; idx += 256) {
    const int rr = idx % NN_ROWS, k = idx / NN_ROWS;
    Ps[k * NN_ROWS + rr] = (rr < rows) ? P[ch.r0 + rr + (int64_t)(poff + k) * ldp] : (T)0;
  }
  for (int idx = tid; idx < kin * NN_MAX; idx += 256) {
    const int j = idx % NN_MAX, k = idx / NN_MAX;
    Cs[k * NN_MAX + j] = (j < kout) ? Cn[k + (int64_t)j * cld] : (T)0;
  }
  __syncthreads();
  const int lane = tid & 31, w = tid >> 5;
  double acc[2][16];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < kin; k0 += 16) {
    const int k1 = (k0 + 16 < kin) ? k0 + 16 : kin;
    T tmp[2][16];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 16; ++j) tmp[i][j] = 0;
    for (int k = k0; k < k1; ++k) {
      const T a0 = Ps[k * NN_ROWS + lane], a1 = Ps[k * NN_ROWS + lane + 32];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const T c = Cs[k * NN_MAX + w * 16 + j];
        tmp[0][j] = fma(a0, c, tmp[0][j]);
        tmp[1][j] = fma(a1, c, tmp[1][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[i][j] += (double)tmp[i][j];
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int col = w * 16 + j;
    if (col >= kout) continue;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int rr = lane + 32 * i;
      if (rr >= rows) continue;
      T* yp = Y + ch.r0 + rr + (int64_t)(yoff + col) * ldy;
      const double v = (double)alpha * acc[i][j];
      *yp = (beta == (T)0) ? (T)v : (T)(v + (double)beta * (double)(*yp));
    }
  }
}

// The FP64 expansion in double-float arithmetic (HM_A32), as k_seg_tn_partial_df:
// inputs cut to hi + lo floats when staged, products by TwoProduct, sums by TwoSum.
// Warp w owns output columns [CJ w, CJ w + CJ) (CJ = 4, 8 or 16 as kout needs), so
// only the columns that cover kout are staged and computed.
template <int CJ>
__global__ __launch_bounds__(256) void k_seg_nn_df(
    const Chunk* __restrict__ chunks, int node0, const double* P, int64_t ldp, int poff_e,
    int poff_o, int kin, const double* __restrict__ C, int64_t cstride, int cld, int cflip,
    double* Y, int64_t ldy, int yoff_e, int yoff_o, int kout, double alpha, double beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int CW = 8 * CJ;                      // staged columns of C
  float* Ph = reinterpret_cast<float*>(smem_raw);  // [NN_MAX][NN_ROWS] each
  float* Pl = Ph + NN_MAX * NN_ROWS;
  float* Ch = Pl + NN_MAX * NN_ROWS;              // [NN_MAX][CW] each
  float* Cl = Ch + NN_MAX * CW;
  const Chunk ch = chunks[blockIdx.x];
  const int rows = (int)(ch.r1 - ch.r0);
  const int poff = (ch.node & 1) ? poff_o : poff_e;
  const int yoff = (ch.node & 1) ? yoff_o : yoff_e;
  const double* Cn = C + (int64_t)((ch.node ^ cflip) - node0) * cstride;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kin * NN_ROWS; idx += 256) {
    const int rr = idx % NN_ROWS, k = idx / NN_ROWS;
    float h, l;
    split_df((rr < rows) ? P[ch.r0 + rr + (int64_t)(poff + k) * ldp] : 0.0, h, l);
    Ph[k * NN_ROWS + rr] = h;
    Pl[k * NN_ROWS + rr] = l;
  }
  for (int idx = tid; idx < kin * CW; idx += 256) {
    const int j = idx % CW, k = idx / CW;
    float h, l;
    split_df((j < kout) ? Cn[k + (int64_t)j * cld] : 0.0, h, l);
    Ch[k * CW + j] = h;
    Cl[k * CW + j] = l;
  }
  __syncthreads();
  const int lane = tid & 31, w = tid >> 5;
  float sh[2][CJ], sl[2][CJ];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < CJ; ++j) { sh[i][j] = 0.f; sl[i][j] = 0.f; }
  for (int k = 0; k < kin; ++k) {
    const float ah[2] = {Ph[k * NN_ROWS + lane], Ph[k * NN_ROWS + lane + 32]};
    const float al[2] = {Pl[k * NN_ROWS + lane], Pl[k * NN_ROWS + lane + 32]};
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      const float chj = Ch[k * CW + w * CJ + j], clj = Cl[k * CW + w * CJ + j];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float p = ah[i] * chj;
        const float e = fmaf(ah[i], chj, -p);
        const float t = fmaf(ah[i], clj, fmaf(al[i], chj, e));
        const float s = sh[i][j] + p;
        const float z = s - sh[i][j];
        const float err = (sh[i][j] - (s - z)) + (p - z);
        sh[i][j] = s;
        sl[i][j] += err + t;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < CJ; ++j) {
    const int col = w * CJ + j;
    if (col >= kout) continue;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int rr = lane + 32 * i;
      if (rr >= rows) continue;
      double* yp = Y + ch.r0 + rr + (int64_t)(yoff + col) * ldy;
      const double v = alpha * ((double)sh[i][j] + (double)sl[i][j]);
      *yp = (beta == 0.0) ? v : v + beta * (*yp);
    }
  }
}

}  // namespace

template <typename T, int TI, int TJ>
void seg_tn_partial_tiled(const Chunk* chunks, int nchunks, const T* A, int64_t lda,
                          int aoff_even, int aoff_odd, int ka, const T* B, int64_t ldb,
                          int boff_even, int boff_odd, int kb, double* partial, cudaStream_t st,
                          bool df) {
  constexpr int LDA = 16 * TI + 1, LDB = 16 * TJ + 1;
  if (sizeof(T) == 8 && df) {
    const size_t smem = 2 * TN_ROWS * (LDA + LDB) * sizeof(float);
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_seg_tn_partial_df<TI, TJ>, done);
    k_seg_tn_partial_df<TI, TJ><<<nchunks, 256, smem, st>>>(
        chunks, (const double*)A, lda, aoff_even, aoff_odd, ka, (const double*)B, ldb, boff_even,
        boff_odd, kb, partial);
  } else {
    const size_t smem = TN_ROWS * (LDA + LDB) * sizeof(T);
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_seg_tn_partial<T, TI, TJ>, done);
    k_seg_tn_partial<T, TI, TJ><<<nchunks, 256, smem, st>>>(
        chunks, A, lda, aoff_even, aoff_odd, ka, B, ldb, boff_even, boff_odd, kb, partial);
  }
}

template <typename T, int TI>
void seg_tn_partial_pick_j(const Chunk* chunks, int nchunks, const T* A, int64_t lda,
                           int aoff_even, int aoff_odd, int ka, const T* B, int64_t ldb,
                           int boff_even, int boff_odd, int kb, double* partial, cudaStream_t st,
                           bool df) {
  switch (tn_tile(kb)) {
    case 2:
      seg_tn_partial_tiled<T, TI, 2>(chunks, nchunks, A, lda, aoff_even, aoff_odd, ka, B, ldb,
                                     boff_even, boff_odd, kb, partial, st, df);
      break;
    case 4:
      seg_tn_partial_tiled<T, TI, 4>(chunks, nchunks, A, lda, aoff_even, aoff_odd, ka, B, ldb,
                                     boff_even, boff_odd, kb, partial, st, df);
      break;
    default:
      seg_tn_partial_tiled<T, TI, 8>(chunks, nchunks, A, lda, aoff_even, aoff_odd, ka, B, ldb,
                                     boff_even, boff_odd, kb, partial, st, df);
  }
}

template <typename T>
void launch_seg_tn(const Chunk* chunks, int nchunks, const int32_t* chunk_begin, int nnodes,
                   int node0, const T* A, int64_t lda, int aoff_even, int aoff_odd, int ka,
                   const T* B, int64_t ldb, int boff_even, int boff_odd, int kb, double* partial,
                   T* out, cudaStream_t st, bool df) {
  count_launches(2);
  (void)node0;
  switch (tn_tile(ka)) {
    case 2:
      seg_tn_partial_pick_j<T, 2>(chunks, nchunks, A, lda, aoff_even, aoff_odd, ka, B, ldb,
                                  boff_even, boff_odd, kb, partial, st, df);
      break;
    case 4:
      seg_tn_partial_pick_j<T, 4>(chunks, nchunks, A, lda, aoff_even, aoff_odd, ka, B, ldb,
                                  boff_even, boff_odd, kb, partial, st, df);
      break;
    default:
      seg_tn_partial_pick_j<T, 8>(chunks, nchunks, A, lda, aoff_even, aoff_odd, ka, B, ldb,
                                  boff_even, boff_odd, kb, partial, st, df);
  }
  const int m = ka * kb;
  dim3 grid((unsigned)((m + 255) / 256), (unsigned)nnodes);
  k_seg_tn_reduce<T><<<grid, 256, 0, st>>>(partial, chunk_begin, ka, kb, out);
}

template <typename T>
void launch_seg_nn(const Chunk* chunks, int nchunks, int node0, const T* P, int64_t ldp,
                   int poff_even, int poff_odd, int kin, const T* C, int64_t cstride, int cld,
                   int cflip, T* Y, int64_t ldy, int yoff_even, int yoff_odd, int kout, T alpha,
                   T beta, cudaStream_t st, bool df) {
  count_launches(1);
  const size_t smem = (size_t)(NN_MAX * NN_ROWS + NN_MAX * NN_MAX) * sizeof(T);
  if (sizeof(T) == 8 && df) {
    auto run = [&](auto kern, int cw) {
      const size_t sm = (size_t)2 * (NN_MAX * NN_ROWS + NN_MAX * cw) * sizeof(float);
      kern<<<nchunks, 256, sm, st>>>(chunks, node0, (const double*)P, ldp, poff_even, poff_odd,
                                     kin, (const double*)C, cstride, cld, cflip, (double*)Y, ldy,
                                     yoff_even, yoff_odd, kout, (double)alpha, (double)beta);
    };
    static std::atomic<uint32_t> d4{0}, d8{0}, d16{0};
    if (kout <= 32) {
      raise_smem_limit((const void*)k_seg_nn_df<4>, d4);
      run(k_seg_nn_df<4>, 32);
    } else if (kout <= 64) {
      raise_smem_limit((const void*)k_seg_nn_df<8>, d8);
      run(k_seg_nn_df<8>, 64);
    } else {
      raise_smem_limit((const void*)k_seg_nn_df<16>, d16);
      run(k_seg_nn_df<16>, 128);
    }
    return;
  }
  static std::atomic<uint32_t> done{0};
  raise_smem_limit((const void*)k_seg_nn<T>, done);
  k_seg_nn<T><<<nchunks, 256, smem, st>>>(chunks, node0, P, ldp, poff_even, poff_odd, kin, C,
                                          cstride, cld, cflip, Y, ldy, yoff_even, yoff_odd, kout,
                                          alpha, beta);
}

template void launch_seg_tn<float>(const Chunk*, int, const int32_t*, int, int, const float*,
                                   int64_t, int, int, int, const float*, int64_t, int, int, int,
                                   double*, float*, cudaStream_t, bool);
template void launch_seg_tn<double>(const Chunk*, int, const int32_t*, int, int, const double*,
                                    int64_t, int, int, int, const double*, int64_t, int, int,
                                    int, double*, double*, cudaStream_t, bool);
template void launch_seg_nn<float>(const Chunk*, int, int, const float*, int64_t, int, int, int,
                                   const float*, int64_t, int, int, float*, int64_t, int, int,
                                   int, float, float, cudaStream_t, bool);
template void launch_seg_nn<double>(const Chunk*, int, int, const double*, int64_t, int, int,
                                    int, const double*, int64_t, int, int, double*, int64_t, int,
                                    int, int, double, double, cudaStream_t, bool);

}  // namespace hm
