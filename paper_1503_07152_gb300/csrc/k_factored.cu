// Factored HODLR apply y = H x (the O(k N log N) product of Sec. 2.8 with
// sibling matrices B = I) and its hand-written adjoint (vector-Jacobian product
// for x, U, V, D; with r = H x - b and scale 2, the gradients of ||H x - b||^2).
//
// Both are HBM-streaming: every factor byte is read once (and every gradient
// byte written once).  Pass 1 reduces t_node = V(I_node)^T x(I_node) (and
// s_node = U(I_node)^T res(I_node) for the adjoint) over 256-row chunks of all
// levels; pass 2 reduces the chunk partials per node in a fixed order; pass 3
// runs one block per leaf: every row of the leaf gathers the contributions of
// its L ancestors' siblings (ancestor of leaf l on level j = l >> (L - j)) and
// of the leaf block D, and, for the adjoint, writes the gradient rows.
#include <atomic>
#include <string>

#include "hm_internal.h"

namespace hm {
namespace {

constexpr int kMaxK = 64;

// partial[chunk][0:k] = V_j(rows)^T x(rows); with second operand pair for the
// adjoint: partial[chunk][k:2k] = U_j(rows)^T res(rows).  Thread t loads row t's k
// factor entries at once (independent, coalesced loads), the products go to
// shared memory (row-major, stride k + 1: conflict-free both ways), thread
// (col, part) sums its 32-row part of a column, and the 8 parts are added.
__global__ __launch_bounds__(256) void k_fact_partial(const FactChunk* __restrict__ ch,
                                                      int64_t n, int k,
                                                      const float* __restrict__ A0,
                                                      const float* __restrict__ v0,
                                                      const float* __restrict__ A1,
                                                      const float* __restrict__ v1,
                                                      float* __restrict__ partial) {
  extern __shared__ float prod[];  // [256][k + 1]
  __shared__ float red[8][2 * kMaxK];
  const FactChunk c = ch[blockIdx.x];
  const int tid = threadIdx.x;
  const int ldp = k + 1;
  const int64_t row = c.r0 + tid;
  const bool live = row < c.r1;
  const int npair = A1 ? 2 : 1;
  const int cl = tid & 31, part = tid >> 5;
  for (int p = 0; p < npair; ++p) {
    const float* A = (p == 0 ? A0 : A1) + (int64_t)(c.level - 1) * n * k;
    const float xv = live ? (p == 0 ? v0 : v1)[row] : 0.f;
#pragma unroll 8
    for (int col = 0; col < k; ++col)
      prod[tid * ldp + col] = live ? A[row + (int64_t)col * n] * xv : 0.f;
    __syncthreads();
    for (int col = cl; col < k; col += 32) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) s += prod[(part * 32 + i) * ldp + col];
      red[part][p * k + col] = s;
    }
    __syncthreads();
  }
  for (int e = tid; e < npair * k; e += 256) {
    float s = 0.f;
    for (int w = 0; w < 8; ++w) s += red[w][e];
    partial[(int64_t)blockIdx.x * npair * k + e] = s;
  }
}

// out[node][e] = sum over the node's chunks (heap ids 2 .. 2^(L+1)-1).  The
// 256 threads form 256 / width groups; group q sums chunks q, q + groups, ...
// and the group sums are added in group order (deterministic).  width <= 128.
__global__ __launch_bounds__(256) void k_fact_reduce(const float* __restrict__ partial,
                                                     const int32_t* __restrict__ fbegin,
                                                     int width, int nnodes_total,
                                                     float* __restrict__ out) {
  __shared__ float sred[256];
  const int node = 2 + blockIdx.x;
  if (node >= nnodes_total) return;  // uniform over the block
  const int c0 = fbegin[node], c1 = fbegin[node + 1];
  const int groups = 256 / width;
  const int t = threadIdx.x, e = t % width, q = t / width;
  float s = 0.f;
  if (q < groups)
    for (int c = c0 + q; c < c1; c += groups) s += partial[(int64_t)c * width + e];
  sred[t] = s;
  __syncthreads();
  if (t < width) {
    float tot = 0.f;
    for (int g = 0; g < groups; ++g) tot += sred[g * width + t];
    out[(int64_t)node * width + t] = tot;
  }
}

// y(I_leaf) = sum_j Uex_j(I_leaf) coef[sib(anc_j)] + op(D_leaf) x(I_leaf); with
// b, also res = y - b
__global__ __launch_bounds__(256) void k_fact_expand(const int64_t* __restrict__ start,
                                                     const int64_t* __restrict__ size, int L,
                                                     int64_t n, int k, int nmax, int width,
                                                     const float* __restrict__ Uex,
                                                     const float* __restrict__ coef,
                                                     const float* __restrict__ D, int trans,
                                                     const float* __restrict__ x,
                                                     float* __restrict__ y,
                                                     const float* __restrict__ b,
                                                     float* __restrict__ res) {
  extern __shared__ float sm[];
  float* cs = sm;                  // L * k coefficients
  float* xs = sm + L * kMaxK;      // leaf slice of x
  float* dt = xs + nmax;           // D^T x for the transposed product
  const int leaf = (1 << L) + blockIdx.x;
  const int64_t s0 = start[leaf];
  const int ns = (int)size[leaf];
  const int tid = threadIdx.x;
  for (int e = tid; e < L * k; e += blockDim.x) {
    const int j = 1 + e / k, col = e % k;
    const int anc = leaf >> (L - j);
    cs[(j - 1) * kMaxK + col] = coef[(int64_t)(anc ^ 1) * width + col];
  }
  for (int m = tid; m < ns; m += blockDim.x) xs[m] = x[s0 + m];
  __syncthreads();
  const float* Dl = D + (int64_t)blockIdx.x * nmax * nmax;
  if (trans) {
    const int lane = tid & 31, warp = tid >> 5;
    for (int i = warp; i < ns; i += blockDim.x >> 5) {
      float v = 0.f;
      for (int m = lane; m < ns; m += 32) v += Dl[m + (int64_t)i * nmax] * xs[m];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) dt[i] = v;
    }
    __syncthreads();
  }
  for (int i = tid; i < ns; i += blockDim.x) {
    const int64_t row = s0 + i;
    float acc = 0.f;
    for (int j = 1; j <= L; ++j) {
      const float* Uj = Uex + (int64_t)(j - 1) * n * k;
      for (int col = 0; col < k; ++col) acc = fmaf(Uj[row + (int64_t)col * n], cs[(j - 1) * kMaxK + col], acc);
    }
    if (trans) {
      acc += dt[i];
    } else {
      for (int m = 0; m < ns; ++m) acc = fmaf(Dl[i + (int64_t)m * nmax], xs[m], acc);
    }
    if (y) y[row] = acc;
    if (b) res[row] = acc - b[row];
  }
}

// Adjoint rows of one leaf.  Per node, coef_t holds t_node = V_j(I_node)^T x and
// coef_s holds s_node = U_j(I_node)^T res, at node * cw (+ the k entries).
__global__ __launch_bounds__(256) void k_fact_adjoint(
    const int64_t* __restrict__ start, const int64_t* __restrict__ size, int L, int64_t n, int k,
    int nmax, const float* __restrict__ U, const float* __restrict__ V,
    const float* __restrict__ D, const float* __restrict__ coef_t,
    const float* __restrict__ coef_s, int cw, const float* __restrict__ x,
    const float* __restrict__ res, float scale, float* __restrict__ gx, float* __restrict__ gU,
    float* __restrict__ gV, float* __restrict__ gD) {
  extern __shared__ float sm[];
  float* ts = sm;                  // t of the sibling per level
  float* ss = sm + L * kMaxK;      // s of the sibling per level
  float* xs = ss + L * kMaxK;
  float* rs = xs + nmax;
  float* dt = rs + nmax;           // D^T res
  const int leaf = (1 << L) + blockIdx.x;
  const int64_t s0 = start[leaf];
  const int ns = (int)size[leaf];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < L * k; e += blockDim.x) {
    const int j = 1 + e / k, col = e % k;
    const int sib = (leaf >> (L - j)) ^ 1;
    ts[(j - 1) * kMaxK + col] = coef_t[(int64_t)sib * cw + col];
    ss[(j - 1) * kMaxK + col] = coef_s[(int64_t)sib * cw + col];
  }
  for (int m = tid; m < ns; m += blockDim.x) {
    xs[m] = x[s0 + m];
    rs[m] = res[s0 + m];
  }
  __syncthreads();
  const float* Dl = D + (int64_t)blockIdx.x * nmax * nmax;
  if (gx) {
    for (int i = warp; i < ns; i += blockDim.x >> 5) {
      float v = 0.f;
      for (int m = lane; m < ns; m += 32) v += Dl[m + (int64_t)i * nmax] * rs[m];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) dt[i] = v;
    }
    __syncthreads();
  }
  for (int i = tid; i < ns; i += blockDim.x) {
    const int64_t row = s0 + i;
    const float xr = xs[i], rr = rs[i];
    float acc = 0.f;
    for (int j = 1; j <= L; ++j) {
      const int64_t base = (int64_t)(j - 1) * n * k;
      for (int col = 0; col < k; ++col) {
        const int64_t off = base + row + (int64_t)col * n;
        if (gx) acc = fmaf(V[off], ss[(j - 1) * kMaxK + col], acc);
        if (gU) gU[off] = scale * rr * ts[(j - 1) * kMaxK + col];
        if (gV) gV[off] = scale * xr * ss[(j - 1) * kMaxK + col];
      }
    }
    if (gx) gx[row] = scale * (acc + dt[i]);
    if (gD) {
      float* gDl = gD + (int64_t)blockIdx.x * nmax * nmax;
      for (int m = 0; m < nmax; ++m)
        gDl[i + (int64_t)m * nmax] = (m < ns) ? scale * rr * xs[m] : 0.f;
    }
  }
  // rows past the leaf's size (a leaf smaller than n_max): zero, so that the
  // whole n_max x n_max block of every leaf is written
  if (gD && ns < nmax) {
    float* gDl = gD + (int64_t)blockIdx.x * nmax * nmax;
    const int pad = nmax - ns;
    for (int e = tid; e < pad * nmax; e += blockDim.x)
      gDl[ns + e % pad + (int64_t)(e / pad) * nmax] = 0.f;
  }
}

}  // namespace

// dynamic shared memory of k_fact_partial (66.5 KB at k = 64: limit raised once)
static size_t fact_partial_smem(int k) {
  static std::atomic<uint32_t> done{0};
  raise_smem_limit((const void*)k_fact_partial, done);
  return sizeof(float) * 256 * (size_t)(k + 1);
}

// dynamic shared memory of the per-leaf kernels: the sibling coefficients of
// every level plus the leaf's slices of x (and res, D^T res); grows with n_max
static size_t fact_leaf_smem(const hm_tree* t, bool adjoint) {
  const size_t nmax = (size_t)t->nmax, L = (size_t)t->L;
  return adjoint ? sizeof(float) * (2 * L * kMaxK + 3 * nmax)
                 : sizeof(float) * (L * kMaxK + 2 * nmax);
}

hm_status factored_check(const hm_tree* t, bool adjoint) {
  int dev = 0, optin = 0;
  HM_CUDA_TRY(cudaGetDevice(&dev));
  HM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t need = fact_leaf_smem(t, adjoint);
  if (need > (size_t)optin) {
    set_error(std::string(adjoint ? "hm_hodlr_factored_adjoint" : "hm_hodlr_factored_apply") +
              ": leaves of " + std::to_string(t->nmax) + " points need " + std::to_string(need) +
              " bytes of shared memory per block; the device allows " + std::to_string(optin));
    return HM_EINVAL;
  }
  static std::atomic<uint32_t> done_e{0}, done_a{0};
  if (adjoint) raise_smem_limit((const void*)k_fact_adjoint, done_a);
  else raise_smem_limit((const void*)k_fact_expand, done_e);
  return HM_OK;
}

size_t factored_scratch_bytes(const hm_tree* t, int k) {
  const size_t nodes = (size_t)1 << (t->L + 1);
  return sizeof(float) * ((size_t)t->n_fchunks * 2 * k + nodes * 2 * k) + 256;
}

void launch_factored_apply(const hm_tree* t, int k, const float* U, const float* V,
                           const float* D, int trans, const float* x, float* y, float* scratch,
                           cudaStream_t st) {
  count_launches(3);
  const int L = t->L;
  const int nodes = 1 << (L + 1);
  float* partial = scratch;
  float* coef = scratch + (size_t)t->n_fchunks * k;
  // t_node = Proj(I_node)^T x with Proj = V (H x) or U (H^T x)
  k_fact_partial<<<t->n_fchunks, 256, fact_partial_smem(k), st>>>(t->d_fchunks, t->n, k, trans ? U : V, x, nullptr,
                                                nullptr, partial);
  k_fact_reduce<<<nodes - 2, 256, 0, st>>>(partial, t->d_fbegin, k, nodes, coef);
  const int nmax = (int)t->nmax;
  const size_t smem = fact_leaf_smem(t, false);
  k_fact_expand<<<1 << L, 256, smem, st>>>(t->d_start, t->d_size, L, t->n, k, nmax, k,
                                           trans ? V : U, coef, D, trans, x, y, nullptr,
                                           nullptr);
}

void launch_factored_adjoint(const hm_tree* t, int k, const float* U, const float* V,
                             const float* D, const float* x, const float* res, float scale,
                             float* gx, float* gU, float* gV, float* gD, float* scratch,
                             cudaStream_t st) {
  count_launches(3);
  const int L = t->L;
  const int nodes = 1 << (L + 1);
  float* partial = scratch;
  float* coef = scratch + (size_t)t->n_fchunks * 2 * k;
  k_fact_partial<<<t->n_fchunks, 256, fact_partial_smem(k), st>>>(t->d_fchunks, t->n, k, V, x, U, res, partial);
  k_fact_reduce<<<nodes - 2, 256, 0, st>>>(partial, t->d_fbegin, 2 * k, nodes, coef);
  const int nmax = (int)t->nmax;
  const size_t smem = fact_leaf_smem(t, true);
  k_fact_adjoint<<<1 << L, 256, smem, st>>>(t->d_start, t->d_size, L, t->n, k, nmax, U, V, D,
                                            coef, coef + k, 2 * k, x, res, scale, gx, gU, gV,
                                            gD);
}

size_t factored_loss_grad_scratch_bytes(const hm_tree* t, int k) {
  const size_t nodes = (size_t)1 << (t->L + 1);
  return sizeof(float) * ((size_t)t->n_fchunks * k + 2 * nodes * k + 2 * (size_t)t->n) + 512;
}

// y = H x, res = y - b and the adjoint at res, with every factor read twice: the
// forward's projections t = V^T x are the adjoint's too, so the adjoint's first
// pass reads U only, and V is read again only for gx.
void launch_factored_loss_grad(const hm_tree* t, int k, const float* U, const float* V,
                               const float* D, const float* x, const float* b, float scale,
                               float* y, float* res, float* gx, float* gU, float* gV, float* gD,
                               float* scratch, cudaStream_t st) {
  count_launches(6);
  const int L = t->L;
  const int nodes = 1 << (L + 1);
  const int nmax = (int)t->nmax;
  float* partial = scratch;
  float* coef_t = partial + (size_t)t->n_fchunks * k;
  float* coef_s = coef_t + (size_t)nodes * k;
  float* tmp = coef_s + (size_t)nodes * k;
  float* yy = y ? y : tmp;
  float* rr = res ? res : tmp + t->n;
  k_fact_partial<<<t->n_fchunks, 256, fact_partial_smem(k), st>>>(t->d_fchunks, t->n, k, V, x,
                                                                   nullptr, nullptr, partial);
  k_fact_reduce<<<nodes - 2, 256, 0, st>>>(partial, t->d_fbegin, k, nodes, coef_t);
  k_fact_expand<<<1 << L, 256, fact_leaf_smem(t, false), st>>>(
      t->d_start, t->d_size, L, t->n, k, nmax, k, U, coef_t, D, 0, x, yy, b, rr);
  k_fact_partial<<<t->n_fchunks, 256, fact_partial_smem(k), st>>>(t->d_fchunks, t->n, k, U, rr,
                                                                   nullptr, nullptr, partial);
  k_fact_reduce<<<nodes - 2, 256, 0, st>>>(partial, t->d_fbegin, k, nodes, coef_s);
  k_fact_adjoint<<<1 << L, 256, fact_leaf_smem(t, true), st>>>(
      t->d_start, t->d_size, L, t->n, k, nmax, U, V, D, coef_t, coef_s, k, x, rr, scale, gx, gU,
      gV, gD);
}

}  // namespace hm
