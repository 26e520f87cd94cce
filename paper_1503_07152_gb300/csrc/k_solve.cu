// Kernels of the HODLR direct solver (api_solve.cu): batched inversion of small
// dense matrices by Gauss-Jordan elimination with partial pivoting, and the
// assembly of the per-parent Woodbury matrices.
#include <algorithm>

#include "hm_internal.h"

namespace hm {
namespace {

// Inverse of every matrix of a batch, one block per matrix.  W holds the
// augmented [A | I] of each matrix, column-major n x 2n (ld n), in global memory
// (L2-resident at these sizes); out[b] receives A^{-1} (n x n, ld n).  A zero
// pivot raises *singular and the step is skipped (the output is then garbage).
template <typename T>
__global__ __launch_bounds__(512) void k_gauss_jordan(T* __restrict__ W, int n,
                                                      T* __restrict__ out,
                                                      int* __restrict__ singular) {
  __shared__ T fcol[256];
  __shared__ double rv[16];
  __shared__ int ri[16];
  __shared__ int piv;
  T* Wb = W + (int64_t)blockIdx.x * n * 2 * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int n2 = 2 * n;
  for (int k = 0; k < n; ++k) {
    // pivot: the largest |A(i, k)|, i >= k (first on ties)
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += blockDim.x) {
      const double a = fabs((double)Wb[i + (int64_t)k * n]);
      if (a > best) { best = a; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int p = n;
      for (int w = 0; w < nw; ++w)
        if (rv[w] > b || (rv[w] == b && ri[w] < p)) { b = rv[w]; p = ri[w]; }
      if (!(b > 0.0) || p >= n) {
        atomicExch(singular, 1);
        p = k;
      }
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != k)
      for (int j = tid; j < n2; j += blockDim.x) {
        const T t = Wb[k + (int64_t)j * n];
        Wb[k + (int64_t)j * n] = Wb[p + (int64_t)j * n];
        Wb[p + (int64_t)j * n] = t;
      }
    __syncthreads();
    const T pv = Wb[k + (int64_t)k * n];
    const T inv = (pv != (T)0) ? (T)1 / pv : (T)0;
    __syncthreads();
    for (int j = tid; j < n2; j += blockDim.x) Wb[k + (int64_t)j * n] *= inv;
    for (int i = tid; i < n; i += blockDim.x) fcol[i] = (i == k) ? (T)0 : Wb[i + (int64_t)k * n];
    __syncthreads();
    // row i -= f_i row k, all i != k (columns k .. 2n - 1: the eliminated
    // columns left of k are already unit vectors and stay so)
    const int cols = n2 - k;
    for (int e = tid; e < n * cols; e += blockDim.x) {
      const int i = e % n, j = k + e / n;
      if (i != k) Wb[i + (int64_t)j * n] -= fcol[i] * Wb[k + (int64_t)j * n];
    }
    __syncthreads();
  }
  T* ob = out + (int64_t)blockIdx.x * n * n;
  for (int e = tid; e < n * n; e += blockDim.x) ob[e] = Wb[(int64_t)n * n + e];
}

// [D_leaf | I] padded to nmax (identity beyond the leaf size), one block per leaf.
template <typename T>
__global__ void k_gj_load_leaves(const T* __restrict__ D, int nmax,
                                 const int64_t* __restrict__ size, int L, T* __restrict__ W) {
  const int leaf = blockIdx.x;
  const int ns = (int)size[(1 << L) + leaf];
  const T* Dl = D + (int64_t)leaf * nmax * nmax;
  T* Wl = W + (int64_t)leaf * nmax * 2 * nmax;
  for (int e = threadIdx.x; e < nmax * 2 * nmax; e += blockDim.x) {
    const int i = e % nmax, j = e / nmax;
    T v;
    if (j < nmax) v = (i < ns && j < ns) ? Dl[i + (int64_t)j * nmax] : (T)(i == j ? 1 : 0);
    else v = (T)(i == j - nmax ? 1 : 0);
    Wl[e] = v;
  }
}

// [[I, P_b], [P_a, I] | I] for every parent p of a level (children a = 2p,
// b = 2p + 1): P holds V_x^T W_x (r x r, ld r) for the children, indexed by
// x - child0.
template <typename T>
__global__ void k_gj_load_woodbury(const T* __restrict__ P, int r, T* __restrict__ W) {
  const int pi = blockIdx.x;  // parent index within its level
  const int n = 2 * r;
  const T* Pa = P + (int64_t)(2 * pi) * r * r;
  const T* Pb = P + (int64_t)(2 * pi + 1) * r * r;
  T* Wp = W + (int64_t)pi * n * 2 * n;
  for (int e = threadIdx.x; e < n * 2 * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    T v;
    if (j >= n) v = (T)(i == j - n ? 1 : 0);
    else if ((i < r) == (j < r)) v = (T)(i == j ? 1 : 0);
    else if (i < r) v = Pb[i + (int64_t)(j - r) * r];  // top right: V_b^T W_b
    else v = Pa[(i - r) + (int64_t)j * r];             // bottom left: V_a^T W_a
    Wp[e] = v;
  }
}

}  // namespace

template <typename T>
void launch_gauss_jordan(T* work, int batch, int n, T* out, int* singular, cudaStream_t st) {
  count_launches(1);
  k_gauss_jordan<T><<<batch, 512, 0, st>>>(work, n, out, singular);
}

template <typename T>
void launch_gj_load_leaves(const T* D, int nmax, const int64_t* d_size, int L, T* work,
                           cudaStream_t st) {
  count_launches(1);
  k_gj_load_leaves<T><<<1 << L, 256, 0, st>>>(D, nmax, d_size, L, work);
}

template <typename T>
void launch_gj_load_woodbury(const T* P, int r, int nparents, T* work, cudaStream_t st) {
  count_launches(1);
  k_gj_load_woodbury<T><<<nparents, 256, 0, st>>>(P, r, work);
}

#define HM_INST(T)                                                                              \
  template void launch_gauss_jordan<T>(T*, int, int, T*, int*, cudaStream_t);                  \
  template void launch_gj_load_leaves<T>(const T*, int, const int64_t*, int, T*, cudaStream_t); \
  template void launch_gj_load_woodbury<T>(const T*, int, int, T*, cudaStream_t);
HM_INST(float)
HM_INST(double)
#undef HM_INST

}  // namespace hm

namespace hm {
namespace {

// Y = alpha A + beta B (column-major n x ncols blocks)
template <typename T>
__global__ void k_axpby(T* __restrict__ Y, int64_t ldy, T alpha, const T* __restrict__ A,
                        int64_t lda, T beta, const T* __restrict__ B, int64_t ldb, int64_t n,
                        int64_t ncols) {
  for (int64_t c = blockIdx.y; c < ncols; c += gridDim.y)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      Y[i + c * ldy] = alpha * A[i + c * lda] + (beta != (T)0 ? beta * B[i + c * ldb] : (T)0);
}

}  // namespace

template <typename T>
void launch_axpby(T* Y, int64_t ldy, T alpha, const T* A, int64_t lda, T beta, const T* B,
                  int64_t ldb, int64_t n, int64_t ncols, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return;
  count_launches(1);
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 1024),
            (unsigned)std::min<int64_t>(ncols, 65535));
  k_axpby<T><<<grid, 256, 0, st>>>(Y, ldy, alpha, A, lda, beta, B, ldb, n, ncols);
}
template void launch_axpby<float>(float*, int64_t, float, const float*, int64_t, float,
                                  const float*, int64_t, int64_t, int64_t, cudaStream_t);
template void launch_axpby<double>(double*, int64_t, double, const double*, int64_t, double,
                                   const double*, int64_t, int64_t, int64_t, cudaStream_t);

}  // namespace hm
