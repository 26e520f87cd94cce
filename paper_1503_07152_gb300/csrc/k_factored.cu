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

// Four consecutive rows of a column: one 16-byte load when `full` (the rows
// lie inside the chunk and are 16-byte aligned), else masked scalar loads.
__device__ __forceinline__ float4 rows4(const float* __restrict__ p, int64_t row0, int64_t r1,
                                        bool full) {
  if (full) return __ldg(reinterpret_cast<const float4*>(p + row0));
  float4 v;
  v.x = row0 < r1 ? p[row0] : 0.f;
  v.y = row0 + 1 < r1 ? p[row0 + 1] : 0.f;
  v.z = row0 + 2 < r1 ? p[row0 + 2] : 0.f;
  v.w = row0 + 3 < r1 ? p[row0 + 3] : 0.f;
  return v;
}

// partial[chunk][0:k] = V_j(rows)^T x(rows); with the second operand pair (the
// two-call adjoint) partial[chunk][k:2k] = U_j(rows)^T res(rows).  Warp w takes
// half (w & 1) of the chunk's 256 rows and the columns w/2, w/2 + 4, ...: lane l
// reads rows 4l .. 4l + 3 of its half of each column as one float4 (512
// contiguous bytes per warp and column, every column's load in flight at once),
// forms the 4-term dot product with the same rows of the vector, and the warp
// adds its 32 lane sums by butterfly shuffles; the two halves are added in
// shared memory.
//
// The per-node sums out[node][0:width] (width = npair k) are formed by the last
// block of each node to finish (cnt[node] counts the node's finished chunks;
// it starts at zero and the last block sets it back to zero): it adds the
// node's chunk partials with 256 / width thread groups (group q takes chunks
// q, q + groups, ...) and then the group sums in group order, a fixed order.
// KM: the largest k the launch serves (32 or 64), which sizes the register
// arrays.
template <int KM>
__global__ __launch_bounds__(256) void k_fact_partial(const FactChunk* __restrict__ ch,
                                                      int64_t n, int k,
                                                      const float* __restrict__ A0,
                                                      const float* __restrict__ v0,
                                                      const float* __restrict__ A1,
                                                      const float* __restrict__ v1, int vec4,
                                                      float* __restrict__ partial,
                                                      const int32_t* __restrict__ fbegin,
                                                      int32_t* __restrict__ cnt,
                                                      float* __restrict__ out) {
  __shared__ float red[2][2 * kMaxK];
  __shared__ float sred[256];
  __shared__ int s_last;
  const FactChunk c = ch[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, half = w & 1;
  const int npair = A1 ? 2 : 1;
  const int width = npair * k;
  const int64_t row0 = c.r0 + half * 128 + lane * 4;
  const bool full = vec4 && row0 + 3 < c.r1;
  for (int p = 0; p < npair; ++p) {
    const float* A = (p == 0 ? A0 : A1) + (int64_t)(c.level - 1) * n * k;
    const float4 xv = rows4(p == 0 ? v0 : v1, row0, c.r1, full);
    float acc[KM / 4];
#pragma unroll
    for (int i = 0; i < KM / 4; ++i) {
      const int col = (w >> 1) + 4 * i;
      float sum = 0.f;
      if (col < k) {  // uniform over the warp
        const float4 a = rows4(A + (int64_t)col * n, row0, c.r1, full);
        sum = fmaf(a.w, xv.w, fmaf(a.z, xv.z, fmaf(a.y, xv.y, a.x * xv.x)));
      }
      acc[i] = sum;
    }
#pragma unroll
    for (int i = 0; i < KM / 4; ++i) {
      if ((w >> 1) + 4 * i >= k) break;  // uniform over the warp
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
      if (lane == 0) red[half][p * k + (w >> 1) + 4 * i] = acc[i];
    }
  }
  __syncthreads();
  for (int e = tid; e < width; e += 256)
    partial[(int64_t)blockIdx.x * width + e] = red[0][e] + red[1][e];
  // per-node sums by the node's last block
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const int nch = fbegin[c.node + 1] - fbegin[c.node];
    s_last = atomicAdd(&cnt[c.node], 1) == nch - 1;
  }
  __syncthreads();
  if (!s_last) return;  // uniform over the block
  __threadfence();
  const int c0 = fbegin[c.node], c1 = fbegin[c.node + 1];
  const int groups = 256 / width;
  const int e = tid % width, q = tid / width;
  float sum = 0.f;
  if (q < groups)
    for (int cc = c0 + q; cc < c1; cc += groups) sum += __ldcg(&partial[(int64_t)cc * width + e]);
  sred[tid] = sum;
  __syncthreads();
  if (tid < width) {
    float tot = 0.f;
    for (int g = 0; g < groups; ++g) tot += sred[g * width + tid];
    out[(int64_t)c.node * width + tid] = tot;
  }
  if (tid == 0) cnt[c.node] = 0;
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

// The float4 path of k_fact_partial needs every chunk to start on a multiple
// of four rows, n a multiple of four (so every column starts 16-byte aligned)
// and 16-byte aligned operands.
static int fact_vec4(const hm_tree* t, const float* A0, const float* v0, const float* A1,
                     const float* v1) {
  auto al = [](const float* p) { return p == nullptr || ((uintptr_t)p & 15) == 0; };
  return t->fvec4 && t->n % 4 == 0 && al(A0) && al(v0) && al(A1) && al(v1) ? 1 : 0;
}

// Scratch layout shared by the launchers: chunk partials, node sums, then one
// counter per heap id (zeroed here on the stream: the pass's last blocks reset
// their counters, so one clear serves every pass of a call).
static int32_t* fact_counters(const hm_tree* t, float* after, cudaStream_t st) {
  int32_t* cnt = reinterpret_cast<int32_t*>(after);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)1 << (t->L + 1)), st);
  return cnt;
}

static void launch_fact_partial(const hm_tree* t, int k, const float* A0, const float* v0,
                                const float* A1, const float* v1, float* partial, int32_t* cnt,
                                float* out, cudaStream_t st) {
  const int vec4 = fact_vec4(t, A0, v0, A1, v1);
  if (k <= 32)
    k_fact_partial<32><<<t->n_fchunks, 256, 0, st>>>(t->d_fchunks, t->n, k, A0, v0, A1, v1, vec4,
                                                     partial, t->d_fbegin, cnt, out);
  else
    k_fact_partial<64><<<t->n_fchunks, 256, 0, st>>>(t->d_fchunks, t->n, k, A0, v0, A1, v1, vec4,
                                                     partial, t->d_fbegin, cnt, out);
}

size_t factored_apply_scratch_bytes(const hm_tree* t, int k) {
  const size_t nodes = (size_t)1 << (t->L + 1);
  return sizeof(float) * ((size_t)t->n_fchunks * k + nodes * k) + sizeof(int32_t) * nodes;
}

size_t factored_scratch_bytes(const hm_tree* t, int k) {
  const size_t nodes = (size_t)1 << (t->L + 1);
  return sizeof(float) * ((size_t)t->n_fchunks * 2 * k + nodes * 2 * k) +
         sizeof(int32_t) * nodes + 256;
}

void launch_factored_apply(const hm_tree* t, int k, const float* U, const float* V,
                           const float* D, int trans, const float* x, float* y, float* scratch,
                           cudaStream_t st) {
  count_launches(2);
  const int L = t->L;
  const int nodes = 1 << (L + 1);
  float* partial = scratch;
  float* coef = scratch + (size_t)t->n_fchunks * k;
  int32_t* cnt = fact_counters(t, coef + (size_t)nodes * k, st);
  // t_node = Proj(I_node)^T x with Proj = V (H x) or U (H^T x)
  const float* P = trans ? U : V;
  launch_fact_partial(t, k, P, x, nullptr, nullptr, partial, cnt, coef, st);
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
  count_launches(2);
  const int L = t->L;
  const int nodes = 1 << (L + 1);
  float* partial = scratch;
  float* coef = scratch + (size_t)t->n_fchunks * 2 * k;
  int32_t* cnt = fact_counters(t, coef + (size_t)nodes * 2 * k, st);
  launch_fact_partial(t, k, V, x, U, res, partial, cnt, coef, st);
  const int nmax = (int)t->nmax;
  const size_t smem = fact_leaf_smem(t, true);
  k_fact_adjoint<<<1 << L, 256, smem, st>>>(t->d_start, t->d_size, L, t->n, k, nmax, U, V, D,
                                            coef, coef + k, 2 * k, x, res, scale, gx, gU, gV,
                                            gD);
}

size_t factored_loss_grad_scratch_bytes(const hm_tree* t, int k) {
  const size_t nodes = (size_t)1 << (t->L + 1);
  return sizeof(float) * ((size_t)t->n_fchunks * k + 2 * nodes * k + 2 * (size_t)t->n) +
         sizeof(int32_t) * nodes + 512;
}

// y = H x, res = y - b and the adjoint at res, with every factor read twice: the
// forward's projections t = V^T x are the adjoint's too, so the adjoint's first
// pass reads U only, and V is read again only for gx.
void launch_factored_loss_grad(const hm_tree* t, int k, const float* U, const float* V,
                               const float* D, const float* x, const float* b, float scale,
                               float* y, float* res, float* gx, float* gU, float* gV, float* gD,
                               float* scratch, cudaStream_t st) {
  count_launches(4);
  const int L = t->L;
  const int nodes = 1 << (L + 1);
  const int nmax = (int)t->nmax;
  float* partial = scratch;
  float* coef_t = partial + (size_t)t->n_fchunks * k;
  float* coef_s = coef_t + (size_t)nodes * k;
  float* tmp = coef_s + (size_t)nodes * k;
  int32_t* cnt = fact_counters(t, tmp + 2 * (size_t)t->n, st);
  float* yy = y ? y : tmp;
  float* rr = res ? res : tmp + t->n;
  launch_fact_partial(t, k, V, x, nullptr, nullptr, partial, cnt, coef_t, st);
  k_fact_expand<<<1 << L, 256, fact_leaf_smem(t, false), st>>>(
      t->d_start, t->d_size, L, t->n, k, nmax, k, U, coef_t, D, 0, x, yy, b, rr);
  launch_fact_partial(t, k, U, rr, nullptr, nullptr, partial, cnt, coef_s, st);
  k_fact_adjoint<<<1 << L, 256, fact_leaf_smem(t, true), st>>>(
      t->d_start, t->d_size, L, t->n, k, nmax, U, V, D, coef_t, coef_s, k, x, rr, scale, gx, gU,
      gV, gD);
}

}  // namespace hm
