// Sampling GEMM of the dense test operator: Y = A X or Y = A^T X with A a
// row-major N x N matrix and X, Y column-major N x ncols blocks (the black-box
// products A Omega / A^* Omega of Fig. "Randomized compression of a HODLR
// matrix").  The test matrices of the sweeps are zero on half of their rows
// (Omega_1 lives on left children, Omega_2 on right children) and the identity
// probe is zero outside one diagonal band, so a pre-pass marks the all-zero
// (K-tile, column-tile) blocks of X and the GEMM skips them: the work and the
// A bytes read follow the nonzero structure of X.
//
// This is the CUDA-core form: 128 x 64 output tile per block of 256 threads,
// 8 x 4 register tile per thread.  In FP32 every K-tile is accumulated in a
// fresh register tile and added to the running sum with Kahan compensation.
#include "hm_internal.h"

namespace hm {
namespace {

constexpr int BM = 128;
constexpr int BN = 64;

template <typename T> struct KTile { static constexpr int BK = 32; };
template <> struct KTile<double> { static constexpr int BK = 16; };

// flags[kt * nct + ct] = 1 iff X(kt*BK .. , ct*BN ..) has a nonzero entry.
template <typename T>
__global__ void k_tile_flags(const T* __restrict__ X, int64_t ldx, int64_t n, int64_t ncols,
                             uint8_t* __restrict__ flags, int nct) {
  constexpr int BK = KTile<T>::BK;
  const int kt = blockIdx.x, ct = blockIdx.y;
  bool nz = false;
  for (int idx = threadIdx.x; idx < BK * BN; idx += blockDim.x) {
    const int k = idx % BK, c = idx / BK;
    const int64_t row = (int64_t)kt * BK + k, col = (int64_t)ct * BN + c;
    if (row < n && col < ncols) nz |= (X[row + col * ldx] != (T)0);
  }
  nz = __syncthreads_or(nz);
  if (threadIdx.x == 0) flags[(int64_t)kt * nct + ct] = nz ? 1 : 0;
}

template <typename T, int TRANS>
__global__ __launch_bounds__(256) void k_dense_gemm(const T* __restrict__ A, int64_t lda,
                                                    int64_t n, int64_t ncols,
                                                    const T* __restrict__ X, int64_t ldx,
                                                    T* __restrict__ Y, int64_t ldy,
                                                    const uint8_t* __restrict__ flags, int nct) {
  constexpr int BK = KTile<T>::BK;
  __shared__ __align__(16) T As[BK][BM + 4];
  __shared__ __align__(16) T Xs[BK][BN + 4];
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int ct = blockIdx.y;
  const int64_t c0 = (int64_t)ct * BN;
  const int tid = threadIdx.x;
  const int rg = tid >> 4, cg = tid & 15;

  T acc[8][4], cmp[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = 0; cmp[i][j] = 0; }

  const int nkt = (int)((n + BK - 1) / BK);
  for (int kt = 0; kt < nkt; ++kt) {
    if (flags && !flags[(int64_t)kt * nct + ct]) continue;  // uniform over the block
    const int64_t k0 = (int64_t)kt * BK;
    // A tile: BM x BK values of op(A)
    if (!TRANS) {
      // element (m, k) = A[(m0 + m) * lda + k0 + k]; lanes run along k
      for (int idx = tid; idx < BM * BK; idx += 256) {
        const int k = idx % BK, m = idx / BK;
        const int64_t row = m0 + m, col = k0 + k;
        As[k][m] = (row < n && col < n) ? A[row * lda + col] : (T)0;
      }
    } else {
      // element (m, k) = A[(k0 + k) * lda + m0 + m]; lanes run along m
      for (int idx = tid; idx < BM * BK; idx += 256) {
        const int m = idx % BM, k = idx / BM;
        const int64_t row = k0 + k, col = m0 + m;
        As[k][m] = (row < n && col < n) ? A[row * lda + col] : (T)0;
      }
    }
    for (int idx = tid; idx < BK * BN; idx += 256) {
      const int k = idx % BK, c = idx / BK;
      const int64_t row = k0 + k, col = c0 + c;
      Xs[k][c] = (row < n && col < ncols) ? X[row + col * ldx] : (T)0;
    }
    __syncthreads();
    T tmp[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) tmp[i][j] = 0;
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      T a[8], x[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][rg * 8 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = Xs[kk][cg * 4 + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) tmp[i][j] = fma(a[i], x[j], tmp[i][j]);
    }
    // running sum: compensated in FP32, plain in FP64
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (sizeof(T) == 4) {
          const T y = tmp[i][j] - cmp[i][j];
          const T t = acc[i][j] + y;
          cmp[i][j] = (t - acc[i][j]) - y;
          acc[i][j] = t;
        } else {
          acc[i][j] += tmp[i][j];
        }
      }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t col = c0 + cg * 4 + j;
    if (col >= ncols) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t row = m0 + rg * 8 + i;
      if (row < n) Y[row + col * ldy] = acc[i][j];
    }
  }
}

// FP32 operator, FP64 samples: every product a * x is formed and summed in FP64
// (an FP32 value converts to FP64 exactly).
template <int TRANS>
__global__ __launch_bounds__(256) void k_dense_gemm_a32(const float* __restrict__ A, int64_t lda,
                                                        int64_t n, int64_t ncols,
                                                        const double* __restrict__ X, int64_t ldx,
                                                        double* __restrict__ Y, int64_t ldy,
                                                        const uint8_t* __restrict__ flags,
                                                        int nct) {
  constexpr int BK = 16;
  __shared__ __align__(16) double As[BK][BM + 2];
  __shared__ __align__(16) double Xs[BK][BN + 2];
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int ct = blockIdx.y;
  const int64_t c0 = (int64_t)ct * BN;
  const int tid = threadIdx.x;
  const int rg = tid >> 4, cg = tid & 15;
  double acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int nkt = (int)((n + BK - 1) / BK);
  for (int kt = 0; kt < nkt; ++kt) {
    if (flags && !flags[(int64_t)kt * nct + ct]) continue;
    const int64_t k0 = (int64_t)kt * BK;
    if (!TRANS) {
      for (int idx = tid; idx < BM * BK; idx += 256) {
        const int k = idx % BK, m = idx / BK;
        const int64_t row = m0 + m, col = k0 + k;
        As[k][m] = (row < n && col < n) ? (double)A[row * lda + col] : 0.0;
      }
    } else {
      for (int idx = tid; idx < BM * BK; idx += 256) {
        const int m = idx % BM, k = idx / BM;
        const int64_t row = k0 + k, col = m0 + m;
        As[k][m] = (row < n && col < n) ? (double)A[row * lda + col] : 0.0;
      }
    }
    for (int idx = tid; idx < BK * BN; idx += 256) {
      const int k = idx % BK, c = idx / BK;
      const int64_t row = k0 + k, col = c0 + c;
      Xs[k][c] = (row < n && col < ncols) ? X[row + col * ldx] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      double a[8], x[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][rg * 8 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = Xs[kk][cg * 4 + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], x[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t col = c0 + cg * 4 + j;
    if (col >= ncols) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t row = m0 + rg * 8 + i;
      if (row < n) Y[row + col * ldy] = acc[i][j];
    }
  }
}

}  // namespace

void launch_dense_gemm_a32(const float* A, int64_t lda, int trans, int64_t n, int64_t ncols,
                           const double* X, int64_t ldx, double* Y, int64_t ldy, uint8_t* flags,
                           cudaStream_t st) {
  count_launches(flags ? 2 : 1);
  constexpr int BK = 16;
  const int nct = (int)((ncols + BN - 1) / BN);
  const int nkt = (int)((n + BK - 1) / BK);
  if (flags) {
    dim3 gf(nkt, nct);
    k_tile_flags<double><<<gf, 256, 0, st>>>(X, ldx, n, ncols, flags, nct);
  }
  dim3 grid((unsigned)((n + BM - 1) / BM), (unsigned)nct);
  if (trans)
    k_dense_gemm_a32<1><<<grid, 256, 0, st>>>(A, lda, n, ncols, X, ldx, Y, ldy, flags, nct);
  else
    k_dense_gemm_a32<0><<<grid, 256, 0, st>>>(A, lda, n, ncols, X, ldx, Y, ldy, flags, nct);
}

template <typename T>
void launch_dense_gemm(const T* A, int64_t lda, int trans, int64_t n, int64_t ncols, const T* X,
                       int64_t ldx, T* Y, int64_t ldy, uint8_t* flags, cudaStream_t st) {
  count_launches(flags ? 2 : 1);
  constexpr int BK = KTile<T>::BK;
  const int nct = (int)((ncols + BN - 1) / BN);
  const int nkt = (int)((n + BK - 1) / BK);
  if (flags) {
    dim3 gf(nkt, nct);
    k_tile_flags<T><<<gf, 256, 0, st>>>(X, ldx, n, ncols, flags, nct);
  }
  dim3 grid((unsigned)((n + BM - 1) / BM), (unsigned)nct);
  if (trans)
    k_dense_gemm<T, 1><<<grid, 256, 0, st>>>(A, lda, n, ncols, X, ldx, Y, ldy, flags, nct);
  else
    k_dense_gemm<T, 0><<<grid, 256, 0, st>>>(A, lda, n, ncols, X, ldx, Y, ldy, flags, nct);
}

int64_t dense_flags_bytes(int64_t n, int64_t ncols, int is_double) {
  (void)is_double;
  const int BK = 16;  // the smallest K tile of any variant
  return ((n + BK - 1) / BK) * ((ncols + BN - 1) / BN);
}

template void launch_dense_gemm<float>(const float*, int64_t, int, int64_t, int64_t,
                                       const float*, int64_t, float*, int64_t, uint8_t*,
                                       cudaStream_t);
template void launch_dense_gemm<double>(const double*, int64_t, int, int64_t, int64_t,
                                        const double*, int64_t, double*, int64_t, uint8_t*,
                                        cudaStream_t);

}  // namespace hm
