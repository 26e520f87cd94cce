// Elementwise and bookkeeping kernels of the compression sweeps:
//  - Gaussian test matrices from Philox4x32-10 + Box-Muller (Sec. 2.5; the
//    Omega_1 / Omega_2 of Fig. "Randomized compression of a HODLR matrix"),
//  - the identity probe of the diagonal extraction (Sec. 3, "Processing the
//    leaves"), scatter of bases into test matrices, sample gathers,
//  - block-diagonal products with the leaf blocks D_tau,
//  - tile kernels of the Frobenius error (Sec. 5), the log-kernel workload
//    generator, and a NaN/Inf detector.
#include <cuda_bf16.h>

#include "hm_internal.h"

namespace hm {
namespace {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Philox4x32 with ten rounds (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo) {
  const double m = (double)hi * 2097152.0 + (double)(lo >> 11);
  return (m + 0.5) * 1.1102230246251565e-16;  // 2^-53
}

// Heap id of the node on `lv` whose index range holds `row` (uniform-depth tree).
__device__ __forceinline__ int node_of_row(const int64_t* __restrict__ start, int lv,
                                           int64_t row) {
  const int64_t* s = start + (1 << lv);
  int lo = 0, hi = (1 << lv) - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s[mid] <= row) lo = mid; else hi = mid - 1;
  }
  return (1 << lv) + lo;
}

template <typename T>
__device__ __forceinline__ T to_sample(double g, bool bf16) {
  if (bf16) {
    const float f = __double2float_rn(g);
    return (T)__bfloat162float(__float2bfloat16_rn(f));
  }
  return (T)g;
}

// X = [Omega_2 | Omega_1] for the parents on `level`: the Gaussian field of the
// level goes to columns [0, r) on right children and [r, 2r) on left children.
template <typename T>
__global__ void k_gauss_fill(T* __restrict__ X, int64_t ldx, int64_t n, int r, int level,
                             uint32_t k0, uint32_t k1, bool bf16,
                             const int64_t* __restrict__ start) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;  // pair of columns 2p, 2p+1
  if (i >= n) return;
  const int node = node_of_row(start, level + 1, i);
  const int on = (node & 1) ? 0 : r;   // nonzero half
  const int off = (node & 1) ? r : 0;  // zero half
  const uint4 w = philox10(make_uint4((uint32_t)i, (uint32_t)p, (uint32_t)level, 0u), k0, k1);
  const double u1 = uniform53(w.x, w.y);
  const double u2 = uniform53(w.z, w.w);
  const double rho = sqrt(-2.0 * log(u1));
  const double theta = 6.283185307179586 * u2;
  const int c0 = 2 * p;
  X[i + (int64_t)(on + c0) * ldx] = to_sample<T>(rho * cos(theta), bf16);
  X[i + (int64_t)(off + c0) * ldx] = (T)0;
  if (c0 + 1 < r) {
    X[i + (int64_t)(on + c0 + 1) * ldx] = to_sample<T>(rho * sin(theta), bf16);
    X[i + (int64_t)(off + c0 + 1) * ldx] = (T)0;
  }
}

template <typename T>
__global__ void k_identity_probe(T* __restrict__ X, int64_t ldx, int64_t n, int nmax,
                                 const int64_t* __restrict__ start, int L) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= n) return;
  const int leaf = node_of_row(start, L, i);
  X[i + (int64_t)c * ldx] = (i - start[leaf] == c) ? (T)1 : (T)0;
}

// Omega_1(I_alpha,:) = U_alpha (left child -> columns [r, 2r)), Omega_2(I_beta,:)
// = U_beta (right child -> columns [0, r)); the other half is zero.
template <typename T>
__global__ void k_scatter_probe(const T* __restrict__ U, int64_t ldu, T* __restrict__ X,
                                int64_t ldx, int64_t n, int r, int lv,
                                const int64_t* __restrict__ start) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  const int node = node_of_row(start, lv, i);
  const int on = (node & 1) ? 0 : r;
  const int off = (node & 1) ? r : 0;
  X[i + (int64_t)(on + j) * ldx] = U[i + (int64_t)j * ldu];
  X[i + (int64_t)(off + j) * ldx] = (T)0;
}

// P(i, j) = Y(i, sample(node) + j): left children read Y_1 (columns [0, r)),
// right children Y_2 (columns [r, 2r)).
template <typename T>
__global__ void k_gather_sample(const T* __restrict__ Y, int64_t ldy, T* __restrict__ P,
                                int64_t ldp, int64_t n, int r, int lv,
                                const int64_t* __restrict__ start) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  const int node = node_of_row(start, lv, i);
  const int off = (node & 1) ? r : 0;
  P[i + (int64_t)j * ldp] = Y[i + (int64_t)(off + j) * ldy];
}

template <typename T>
__global__ void k_extract_diag(const T* __restrict__ Y, int64_t ldy, T* __restrict__ D,
                               int nmax, const int64_t* __restrict__ start,
                               const int64_t* __restrict__ size, int L) {
  const int leaf = blockIdx.y;  // 0-based leaf index
  const int node = (1 << L) + leaf;
  const int64_t s = start[node];
  const int ns = (int)size[node];
  T* Dl = D + (int64_t)leaf * nmax * nmax;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nmax * nmax;
       idx += gridDim.x * blockDim.x) {
    const int i = idx % nmax, c = idx / nmax;
    Dl[idx] = (i < ns && c < ns) ? Y[s + i + (int64_t)c * ldy] : (T)0;
  }
}

// Y(I_t, c) += sum_j op(D_t)(i, j) X(I_t(j), c); one block per (leaf, 64-row tile, column).
template <typename T>
__global__ void k_blockdiag_apply(const T* __restrict__ D, int nmax, int trans,
                                  const T* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                  int64_t ldy, const int64_t* __restrict__ start,
                                  const int64_t* __restrict__ size, int L) {
  extern __shared__ unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  const int leaf = blockIdx.x;
  const int c = blockIdx.y;
  const int node = (1 << L) + leaf;
  const int64_t s = start[node];
  const int ns = (int)size[node];
  const T* Dl = D + (int64_t)leaf * nmax * nmax;
  for (int j = threadIdx.x; j < ns; j += blockDim.x) xs[j] = X[s + j + (int64_t)c * ldx];
  __syncthreads();
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    T acc = 0;
    if (!trans) {
      for (int j = 0; j < ns; ++j) acc += Dl[i + (int64_t)j * nmax] * xs[j];
    } else {
      for (int j = 0; j < ns; ++j) acc += Dl[j + (int64_t)i * nmax] * xs[j];
    }
    Y[s + i + (int64_t)c * ldy] += acc;
  }
}

template <typename T>
__global__ void k_fill(T* p, int64_t count, T v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

template <typename T>
__global__ void k_copy_cols(const T* __restrict__ src, int64_t lds, T* __restrict__ dst,
                            int64_t ldd, int64_t rows) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (i < rows) dst[i + c * ldd] = src[i + c * lds];
}

template <typename T>
__global__ void k_identity_cols(T* __restrict__ Y, int64_t ldy, int64_t n, int64_t c0) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (i < n) Y[i + c * ldy] = (i == c0 + c) ? (T)1 : (T)0;
}

// A row-major, Ac column-major (n x w); accumulates sum (A - Ac)^2 and sum A^2.
template <typename T, typename TC>
__global__ void k_frob_tile(const T* __restrict__ A, int64_t lda, const TC* __restrict__ Ac,
                            int64_t ldc, int64_t n, int64_t c0, int64_t w,
                            double* __restrict__ acc) {
  __shared__ double red[2][32];
  double d2 = 0.0, a2 = 0.0;
  const int64_t total = n * w;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / w, c = idx % w;  // consecutive threads along a row of A
    const double a = (double)A[i * lda + c0 + c];
    const double d = a - (double)Ac[i + c * ldc];
    d2 += d * d;
    a2 += a * a;
  }
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_down_sync(0xffffffffu, d2, o);
    a2 += __shfl_down_sync(0xffffffffu, a2, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { red[0][wid] = d2; red[1][wid] = a2; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    d2 = lane < nw ? red[0][lane] : 0.0;
    a2 = lane < nw ? red[1][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      d2 += __shfl_down_sync(0xffffffffu, d2, o);
      a2 += __shfl_down_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) { atomicAdd(acc, d2); atomicAdd(acc + 1, a2); }
  }
}

template <typename T>
__global__ void k_nonfinite(const T* __restrict__ p, int64_t count, int32_t* flag) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite((double)p[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

// log |x_i - x_j| on the ellipse (cos t, 0.5 sin t), t = 2 pi i / n; 1 on the diagonal.
__global__ void k_gen_log_kernel(float* __restrict__ A, int64_t n, int64_t lda) {
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    const double ti = 6.283185307179586 * (double)i / (double)n;
    const double xi = cos(ti), yi = 0.5 * sin(ti);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
      const double tj = 6.283185307179586 * (double)j / (double)n;
      const double dx = xi - cos(tj), dy = yi - 0.5 * sin(tj);
      A[i * lda + j] = (i == j) ? 1.0f : __double2float_rn(log(sqrt(dx * dx + dy * dy)));
    }
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <typename T>
void launch_gauss_fill(T* X, int64_t ldx, int64_t n, int r, int level, uint64_t seed, bool bf16,
                       const int64_t* d_start, int L, cudaStream_t st) {
  count_launches(1);
  (void)L;
  dim3 grid(blocks_for(n, 256), (unsigned)((r + 1) / 2));
  k_gauss_fill<T><<<grid, 256, 0, st>>>(X, ldx, n, r, level, (uint32_t)(seed & 0xffffffffu),
                                         (uint32_t)(seed >> 32), bf16, d_start);
}

template <typename T>
void launch_identity_probe(T* X, int64_t ldx, int64_t n, int nmax, const int64_t* d_start, int L,
                           cudaStream_t st) {
  count_launches(1);
  dim3 grid(blocks_for(n, 256), (unsigned)nmax);
  k_identity_probe<T><<<grid, 256, 0, st>>>(X, ldx, n, nmax, d_start, L);
}

template <typename T>
void launch_scatter_probe(const T* U, int64_t ldu, T* X, int64_t ldx, int64_t n, int r,
                          int level_nodes, const int64_t* d_start, int L, cudaStream_t st) {
  count_launches(1);
  (void)L;
  dim3 grid(blocks_for(n, 256), (unsigned)r);
  k_scatter_probe<T><<<grid, 256, 0, st>>>(U, ldu, X, ldx, n, r, level_nodes, d_start);
}

template <typename T>
void launch_gather_sample(const T* Y, int64_t ldy, T* P, int64_t ldp, int64_t n, int r,
                          int level_nodes, const int64_t* d_start, int L, cudaStream_t st) {
  count_launches(1);
  (void)L;
  dim3 grid(blocks_for(n, 256), (unsigned)r);
  k_gather_sample<T><<<grid, 256, 0, st>>>(Y, ldy, P, ldp, n, r, level_nodes, d_start);
}

template <typename T>
void launch_extract_diag(const T* Y, int64_t ldy, T* D, int nmax, const int64_t* d_start,
                         const int64_t* d_size, int L, cudaStream_t st) {
  count_launches(1);
  dim3 grid(blocks_for((int64_t)nmax * nmax, 256) < 64 ? blocks_for((int64_t)nmax * nmax, 256)
                                                       : 64,
            1u << L);
  k_extract_diag<T><<<grid, 256, 0, st>>>(Y, ldy, D, nmax, d_start, d_size, L);
}

template <typename T>
void launch_blockdiag_apply(const T* D, int nmax, int trans, const T* X, int64_t ldx, T* Y,
                            int64_t ldy, int64_t ncols, const int64_t* d_start,
                            const int64_t* d_size, int L, cudaStream_t st) {
  count_launches(1);
  dim3 grid(1u << L, (unsigned)ncols);
  k_blockdiag_apply<T><<<grid, 256, nmax * sizeof(T), st>>>(D, nmax, trans, X, ldx, Y, ldy,
                                                            d_start, d_size, L);
}

template <typename T>
void launch_fill(T* p, int64_t count, T v, cudaStream_t st) {
  if (count <= 0) return;
  count_launches(1);
  unsigned g = blocks_for(count, 256);
  k_fill<T><<<g > 4096 ? 4096 : g, 256, 0, st>>>(p, count, v);
}

template <typename T>
void launch_copy_cols(const T* src, int64_t lds, T* dst, int64_t ldd, int64_t rows, int64_t cols,
                      cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  count_launches(1);
  dim3 grid(blocks_for(rows, 256), (unsigned)cols);
  k_copy_cols<T><<<grid, 256, 0, st>>>(src, lds, dst, ldd, rows);
}

template <typename T>
void launch_identity_cols(T* Y, int64_t ldy, int64_t n, int64_t c0, int64_t w, cudaStream_t st) {
  count_launches(1);
  dim3 grid(blocks_for(n, 256), (unsigned)w);
  k_identity_cols<T><<<grid, 256, 0, st>>>(Y, ldy, n, c0);
}

template <typename T>
void launch_frob_tile(const T* A, int64_t lda, const T* Ac, int64_t ldc, int64_t n, int64_t c0,
                      int64_t w, double* acc, cudaStream_t st) {
  count_launches(1);
  unsigned g = blocks_for(n * w, 256);
  k_frob_tile<T, T><<<g > 2048 ? 2048 : g, 256, 0, st>>>(A, lda, Ac, ldc, n, c0, w, acc);
}

void launch_frob_tile_a32(const float* A, int64_t lda, const double* Ac, int64_t ldc, int64_t n,
                          int64_t c0, int64_t w, double* acc, cudaStream_t st) {
  count_launches(1);
  unsigned g = blocks_for(n * w, 256);
  k_frob_tile<float, double><<<g > 2048 ? 2048 : g, 256, 0, st>>>(A, lda, Ac, ldc, n, c0, w, acc);
}

int32_t nonfinite_check_launch(const void* p, int64_t count, int is_double, int32_t* flag,
                               cudaStream_t st) {
  if (count <= 0) return 0;
  count_launches(1);
  unsigned g = blocks_for(count, 256);
  if (g > 2048) g = 2048;
  if (is_double) k_nonfinite<double><<<g, 256, 0, st>>>((const double*)p, count, flag);
  else k_nonfinite<float><<<g, 256, 0, st>>>((const float*)p, count, flag);
  return 0;
}

void launch_gen_log_kernel(float* A, int64_t n, int64_t lda, cudaStream_t st) {
  count_launches(1);
  unsigned gx = blocks_for(n, 256);
  if (gx > 64) gx = 64;
  dim3 grid(gx, (unsigned)(n < 32768 ? n : 32768));
  k_gen_log_kernel<<<grid, 256, 0, st>>>(A, n, lda);
}

#define HM_INST(T)                                                                          \
  template void launch_gauss_fill<T>(T*, int64_t, int64_t, int, int, uint64_t, bool,        \
                                     const int64_t*, int, cudaStream_t);                    \
  template void launch_identity_probe<T>(T*, int64_t, int64_t, int, const int64_t*, int,    \
                                         cudaStream_t);                                     \
  template void launch_scatter_probe<T>(const T*, int64_t, T*, int64_t, int64_t, int, int,  \
                                        const int64_t*, int, cudaStream_t);                 \
  template void launch_gather_sample<T>(const T*, int64_t, T*, int64_t, int64_t, int, int,  \
                                        const int64_t*, int, cudaStream_t);                 \
  template void launch_extract_diag<T>(const T*, int64_t, T*, int, const int64_t*,          \
                                       const int64_t*, int, cudaStream_t);                  \
  template void launch_blockdiag_apply<T>(const T*, int, int, const T*, int64_t, T*,        \
                                          int64_t, int64_t, const int64_t*, const int64_t*, \
                                          int, cudaStream_t);                               \
  template void launch_fill<T>(T*, int64_t, T, cudaStream_t);                               \
  template void launch_copy_cols<T>(const T*, int64_t, T*, int64_t, int64_t, int64_t,       \
                                    cudaStream_t);                                          \
  template void launch_identity_cols<T>(T*, int64_t, int64_t, int64_t, int64_t,            \
                                        cudaStream_t);                                      \
  template void launch_frob_tile<T>(const T*, int64_t, const T*, int64_t, int64_t, int64_t, \
                                    int64_t, double*, cudaStream_t);
HM_INST(float)
HM_INST(double)
#undef HM_INST

}  // namespace hm
