// Sampling GEMM of the dense test operator on the 5th-generation tensor cores
// (tcgen05 + TMEM), FP32 operator, FP32 samples: Y = op(A) X.
//
// Split precision: every FP32 value a of A is split into three BF16 slices
// a = a_h + a_m + a_l (exact for normal FP32 values); X is split the same way
// by a pre-pass.  The products of the slice pairs whose order is at most 2
// (h*h, m*h, l*h, h*m, m*m, h*l) are issued as BF16 MMAs with FP32 accumulation
// in TMEM; a product of two BF16 slices is exact in FP32.  When X holds BF16
// values (the Gaussian test matrices of the sweeps) its m and l slices are zero
// and only the three products with x_h are issued.
//
// Block: 128 rows of op(A) x 64 columns of X, ten warps in four roles.
//   warp 9 (one lane): TMA loads of the FP32 tile of A (128 x 64 for Y = A X,
//     64 x 128 for Y = A^T X) into a ring of raw stages;
//   warps 0-3: split each raw tile into three BF16 slices stored as K-major
//     tiles with the 128-byte swizzle (the transpose of A^T is taken here), and
//     one lane loads the matching pre-split X slices by TMA (128-byte swizzle);
//   warp 4: allocates TMEM; one lane issues the MMAs;
//   warps 5-8: drain the accumulators into compensated FP32 sums in registers
//     and write Y.
// The tensor cores round (toward zero) whenever they add into an FP32
// accumulator, so the accumulators are kept short: every 64-wide K tile gets a
// fresh pair of accumulators, one for the leading product h*h and one for the
// five correction products (2^-8 smaller, so their rounding is negligible).
// Two pairs alternate, so the drain overlaps the MMAs of the next tile.  All-zero
// K tiles of X are skipped (flags from the pre-pass), so the A bytes read follow
// the nonzero structure of X.  When no tile of the block's columns of X needs
// the m and l slices, the X stage area shrinks to one slice and a third raw
// stage of A is kept in flight.
//
// Every wait on an mbarrier is bounded; on timeout the block raises an error
// flag, writes NaN to its outputs, waits (bounded) for its own TMA copies still
// in flight and leaves through the common exit path.  TMEM is released unless
// the wait for the block's own MMAs itself timed out (freeing it under running
// MMAs would be worse than leaking it).
#include <atomic>

#include "tc_util.cuh"

namespace hm {
namespace {

using namespace tc;

constexpr int TM = 128, TN = 64, TK = 64;
constexpr int A_SLICE = TM * TK * 2;    // bytes of one BF16 slice tile of A
constexpr int B_SLICE = TN * TK * 2;    // bytes of one BF16 slice tile of X
constexpr int RAW_BYTES = TM * TK * 4;  // one FP32 tile of A as loaded by TMA
constexpr int SSTAGES = 2;              // split (MMA operand) stages
constexpr int MAX_RAW = 3;              // raw stages with one X slice; two with three
// both layouts need the same room: 3 raw + 2 x (3 A + 1 X) = 2 raw + 2 x (3 A + 3 X)
constexpr int LAYOUT_BYTES = 3 * RAW_BYTES + SSTAGES * (3 * A_SLICE + B_SLICE);
static_assert(LAYOUT_BYTES == 2 * RAW_BYTES + SSTAGES * (3 * A_SLICE + 3 * B_SLICE), "layout");
constexpr int NCONV = 128, NTHREADS = 320;
constexpr uint32_t TMEM_COLS = 4 * TN;  // two (leading, correction) pairs

// Three-way BF16 split of an FP32 value.
__device__ __forceinline__ void split3(float a, __nv_bfloat16& h, __nv_bfloat16& m,
                                      __nv_bfloat16& l) {
  h = __float2bfloat16_rn(a);
  const float r1 = a - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(m);
  l = __float2bfloat16_rn(r2);
}

// The same split for two values at once; results as packed BF16 pairs.
__device__ __forceinline__ void split3x2(float a, float b, uint32_t& h, uint32_t& m, uint32_t& l) {
  const __nv_bfloat162 hh = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(hh);
  const float ra = a - hf.x, rb = b - hf.y;
  const __nv_bfloat162 mm = __floats2bfloat162_rn(ra, rb);
  const float2 mf = __bfloat1622float2(mm);
  const __nv_bfloat162 ll = __floats2bfloat162_rn(ra - mf.x, rb - mf.y);
  h = *reinterpret_cast<const uint32_t*>(&hh);
  m = *reinterpret_cast<const uint32_t*>(&mm);
  l = *reinterpret_cast<const uint32_t*>(&ll);
}

// X (FP32, column-major n x ncols) -> three BF16 slices, layout
// Xs[((ct * 3 + s) * 64 + c) * kpad + k]; flags[kt * nct + ct] = bit s set when
// slice s of the (kt, ct) tile has a nonzero entry.
__global__ void k_split_x(const float* __restrict__ X, int64_t ldx, int64_t n, int64_t ncols,
                          int64_t kpad, int nct, __nv_bfloat16* __restrict__ Xs,
                          uint8_t* __restrict__ flags) {
  const int kt = blockIdx.x, ct = blockIdx.y;
  int mask = 0;
  for (int idx = threadIdx.x; idx < TK * TN; idx += blockDim.x) {
    const int k = idx % TK, c = idx / TK;
    const int64_t row = (int64_t)kt * TK + k, col = (int64_t)ct * TN + c;
    const float v = (row < n && col < ncols) ? X[row + col * ldx] : 0.f;
    __nv_bfloat16 h, m, l;
    split3(v, h, m, l);
    const int64_t base = (int64_t)ct * 3 * TN;
    Xs[(base + c) * kpad + row] = h;
    Xs[(base + TN + c) * kpad + row] = m;
    Xs[(base + 2 * TN + c) * kpad + row] = l;
    mask |= (__bfloat162float(h) != 0.f ? 1 : 0) | (__bfloat162float(m) != 0.f ? 2 : 0) |
            (__bfloat162float(l) != 0.f ? 4 : 0);
  }
  __shared__ int red[8];
  for (int o = 16; o > 0; o >>= 1) mask |= __shfl_xor_sync(0xffffffffu, mask, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mask;
  __syncthreads();
  if (threadIdx.x == 0) {
    int mm = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm |= red[w];
    flags[(int64_t)kt * nct + ct] = (uint8_t)mm;
  }
}

template <int TRANS>
__global__ __launch_bounds__(NTHREADS, 1) void k_gemm_tc(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX, int64_t n,
    int64_t ncols, const uint8_t* __restrict__ flags, float* __restrict__ Y, int64_t ldy,
    int* __restrict__ err, long long poll_limit) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t raw_full[MAX_RAW], raw_empty[MAX_RAW], st_full[SSTAGES],
      x_full[SSTAGES], st_empty[SSTAGES], acc_full[2], acc_empty[2], bar_final;
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ct = blockIdx.x, mt = blockIdx.y, nct = gridDim.x;
  const int64_t m0 = (int64_t)mt * TM;
  const int nkt = (int)((n + TK - 1) / TK);
  // 1024-byte aligned buffers (the 128-byte swizzle repeats every 1024 bytes)
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sbase = smem_raw + (base - raw);

  if (tid == 0) {
    abort_flag = 0;
    for (int i = 0; i < MAX_RAW; ++i) {
      mbar_init(smem_u32(&raw_full[i]), 1);
      mbar_init(smem_u32(&raw_empty[i]), NCONV);
    }
    for (int i = 0; i < SSTAGES; ++i) {
      mbar_init(smem_u32(&st_full[i]), NCONV);
      mbar_init(smem_u32(&x_full[i]), 1);
      mbar_init(smem_u32(&st_empty[i]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), 128);
    }
    mbar_init(smem_u32(&bar_final), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the list of active K tiles is the same for every role
  auto active = [&](int kt) -> int { return flags[(int64_t)kt * nct + ct]; };
  // does any K tile of this block's columns need the m or l slice of X?
  int need_ml = 0;
  for (int kt = tid; kt < nkt; kt += NTHREADS) need_ml |= active(kt) & 6;
  tc_fence_before();
  need_ml = __syncthreads_or(need_ml);
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;
  const int nraw = need_ml ? 2 : 3;
  const uint32_t stage_bytes = 3 * A_SLICE + (need_ml ? 3 : 1) * B_SLICE;
  const uint32_t raw_addr0 = base, stage_addr0 = base + (uint32_t)nraw * RAW_BYTES;

  if (warp == 9) {
    // ---------------------------------------------------------- TMA of A
    if (lane == 0) {
      int it = 0;
      for (int kt = 0; kt < nkt; ++kt) {
        if (!active(kt)) continue;
        const int rs = it % nraw;
        if (!mbar_wait(smem_u32(&raw_empty[rs]), ((it / nraw) & 1) ^ 1, &abort_flag, poll_limit)) break;
        mbar_arrive_tx(smem_u32(&raw_full[rs]), RAW_BYTES);
        const int k0 = kt * TK;
        if (!TRANS)
          tma_load_2d(raw_addr0 + rs * RAW_BYTES, &tmA, k0, (int)m0, smem_u32(&raw_full[rs]));
        else
          tma_load_2d(raw_addr0 + rs * RAW_BYTES, &tmA, (int)m0, k0, smem_u32(&raw_full[rs]));
        ++it;
      }
      // the copies still in flight land before the block leaves
      for (int j = (it > nraw ? it - nraw : 0); j < it; ++j)
        mbar_wait_drain(smem_u32(&raw_full[j % nraw]), (j / nraw) & 1);
    }
  } else if (warp < 4) {
    // ---------------------------------------------------------- split A, TMA of X
    int it = 0, xissued = 0;
    for (int kt = 0; kt < nkt && !abort_flag; ++kt) {
      const int fl = active(kt);
      if (!fl) continue;
      const int rs = it % nraw, s = it % SSTAGES;
      if (!mbar_wait(smem_u32(&st_empty[s]), ((it / SSTAGES) & 1) ^ 1, &abort_flag, poll_limit)) break;
      const uint32_t st = stage_addr0 + (uint32_t)s * stage_bytes;
      if (tid == 0) {
        const uint32_t nsl = (uint32_t)__popc(fl & 7);
        mbar_arrive_tx(smem_u32(&x_full[s]), nsl * B_SLICE);
        for (int sl = 0; sl < 3; ++sl)
          if (fl & (1 << sl))
            tma_load_2d(st + 3 * A_SLICE + sl * B_SLICE, &tmX, kt * TK, (ct * 3 + sl) * TN,
                        smem_u32(&x_full[s]));
        xissued = it + 1;
      }
      if (!mbar_wait(smem_u32(&raw_full[rs]), (it / nraw) & 1, &abort_flag, poll_limit)) break;
      const unsigned char* rw = sbase + (size_t)(raw_addr0 - base) + (size_t)rs * RAW_BYTES;
      unsigned char* sp = sbase + (st - base);
      if (!TRANS) {
        // raw: [128 rows][64 k] FP32; a pass covers 8 rows, 16 float4 per row
#pragma unroll 4
        for (int p = 0; p < 16; ++p) {
          const int f = p * NCONV + tid, m = f >> 4, k4 = f & 15;
          const float4 v = *reinterpret_cast<const float4*>(rw + m * 256 + k4 * 16);
          uint32_t h0, m0_, l0, h1, m1_, l1;
          split3x2(v.x, v.y, h0, m0_, l0);
          split3x2(v.z, v.w, h1, m1_, l1);
          const uint32_t off = sw_off(m, k4 >> 1) + (uint32_t)((k4 & 1) * 8);
          *reinterpret_cast<uint2*>(sp + off) = make_uint2(h0, h1);
          *reinterpret_cast<uint2*>(sp + A_SLICE + off) = make_uint2(m0_, m1_);
          *reinterpret_cast<uint2*>(sp + 2 * A_SLICE + off) = make_uint2(l0, l1);
        }
      } else {
        // raw: [64 k][128 m] FP32; thread m gathers its column, 8 k at a time
        const int m = tid;
#pragma unroll 2
        for (int q = 0; q < 8; ++q) {
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e)
            v[e] = *reinterpret_cast<const float*>(rw + ((q * 8 + e) * TM + m) * 4);
          uint32_t h[4], md[4], l[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split3x2(v[2 * e], v[2 * e + 1], h[e], md[e], l[e]);
          const uint32_t off = sw_off(m, q);
          *reinterpret_cast<uint4*>(sp + off) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>(sp + A_SLICE + off) = make_uint4(md[0], md[1], md[2], md[3]);
          *reinterpret_cast<uint4*>(sp + 2 * A_SLICE + off) = make_uint4(l[0], l[1], l[2], l[3]);
        }
      }
      fence_proxy_async();
      mbar_arrive(smem_u32(&raw_empty[rs]));
      mbar_arrive(smem_u32(&st_full[s]));
      ++it;
    }
    if (tid == 0)
      for (int j = (xissued > SSTAGES ? xissued - SSTAGES : 0); j < xissued; ++j)
        mbar_wait_drain(smem_u32(&x_full[j % SSTAGES]), (j / SSTAGES) & 1);
  } else if (warp == 4) {
    // ---------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32();
      int it = 0;
      bool ok = true;
      for (int kt = 0; kt < nkt && ok; ++kt) {
        const int fl = active(kt);
        if (!fl) continue;
        const int b = it & 1, s = it % SSTAGES;
        ok = mbar_wait(smem_u32(&acc_empty[b]), ((it >> 1) & 1) ^ 1, &abort_flag, poll_limit) &&
             mbar_wait(smem_u32(&st_full[s]), (it / SSTAGES) & 1, &abort_flag, poll_limit) &&
             mbar_wait(smem_u32(&x_full[s]), (it / SSTAGES) & 1, &abort_flag, poll_limit);
        if (!ok) break;
        tc_fence_after();
        const uint32_t st = stage_addr0 + (uint32_t)s * stage_bytes;
        const uint32_t d_lead = tmem + (uint32_t)(b * 2 * TN), d_corr = d_lead + TN;
        uint32_t acc_lead = 0u, acc_corr = 0u;  // the first MMA into each overwrites
#pragma unroll
        for (int kk = 0; kk < TK / 16; ++kk) {
#pragma unroll
          for (int p = 0; p < 6; ++p) {
            const int sa = (p < 3) ? p : (p < 5 ? p - 3 : 0);
            const int sb = (p < 3) ? 0 : (p < 5 ? 1 : 2);
            if (!(fl & (1 << sb))) continue;
            const uint64_t ad = sw128_desc(st + sa * A_SLICE + kk * 32);
            const uint64_t bd = sw128_desc(st + 3 * A_SLICE + sb * B_SLICE + kk * 32);
            if (p == 0) {
              mma_bf16(d_lead, ad, bd, idesc, acc_lead);
              acc_lead = 1u;
            } else {
              mma_bf16(d_corr, ad, bd, idesc, acc_corr);
              acc_corr = 1u;
            }
          }
        }
        mma_commit(smem_u32(&st_empty[s]));
        mma_commit(smem_u32(&acc_full[b]));
        ++it;
      }
      // every MMA issued by this thread has completed before TMEM can be released
      mma_commit(smem_u32(&bar_final));
      if (!mbar_wait_drain(smem_u32(&bar_final), 0)) {
        // even the full-limit wait (which ignores the other roles' abort) gave
        // up: leave TMEM allocated rather than free it under running MMAs (the
        // error flag reports the block)
        abort_flag = 2;
      }
    }
  } else {
    // ---------------------------------------------------------- drain / epilogue
    const int q4 = warp & 3;  // TMEM lane quarter of this warp
    const int r = q4 * 32 + lane;
    float acc[TN], cmp[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) { acc[j] = 0.f; cmp[j] = 0.f; }
    // per active K tile: acc += lead + corr, compensated; the correction term is
    // folded into the compensation (it is far below the leading term)
    int it = 0;
    for (int kt = 0; kt < nkt; ++kt) {
      const int fl = active(kt);
      if (!fl) continue;
      const int b = it & 1;
      if (!mbar_wait(smem_u32(&acc_full[b]), (it >> 1) & 1, &abort_flag, poll_limit)) break;
      tc_fence_after();
      const uint32_t t_lane = (uint32_t)(q4 * 32) << 16;
      const uint32_t t_lead = tmem + t_lane + (uint32_t)(b * 2 * TN), t_corr = t_lead + TN;
      // the leading accumulator is written only when the h slice of X is present
      const bool has_lead = (fl & 1) != 0;
#pragma unroll
      for (int g = 0; g < TN / 16; ++g) {
        float d0[16], d1[16];
        tmem_ld16(t_corr + (uint32_t)(g * 16), d1);
        if (has_lead) {
          tmem_ld16(t_lead + (uint32_t)(g * 16), d0);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) d0[j] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float& a = acc[g * 16 + j];
          float& c = cmp[g * 16 + j];
          const float y = d0[j] - c;
          const float t = a + y;
          c = ((t - a) - y) - d1[j];
          a = t;
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&acc_empty[b]));
      ++it;
    }
    const int64_t grow = m0 + r;
    const bool bad = abort_flag != 0;
    if (grow < n) {
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t col = (int64_t)ct * TN + j;
        if (col < ncols)
          Y[grow + col * ldy] = bad ? __int_as_float(0x7fc00000)
                                    : (float)((double)acc[j] - (double)cmp[j]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (abort_flag && tid == 0) atomicExch(err, 1);
  if (warp == 4 && abort_flag != 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

}  // namespace

size_t gemm_tc_smem_bytes() { return (size_t)LAYOUT_BYTES + 1024; }

int64_t gemm_tc_xs_elems(int64_t n, int64_t ncols) {
  const int64_t kpad = ((n + TK - 1) / TK) * TK;
  const int64_t nct = (ncols + TN - 1) / TN;
  return nct * 3 * TN * kpad;
}

bool gemm_tc_supported(const float* A, int64_t lda, int64_t n) {
  // TMA: 16-byte aligned base and row stride; rows at least one tile long
  return n >= TM && n < ((int64_t)1 << 31) && (lda % 4) == 0 &&
         (((uintptr_t)A) & 15) == 0;
}

PFN_cuTensorMapEncodeTiled_v12000 tc::encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  }();
  return fn;
}

int launch_gemm_tc(const float* A, int64_t lda, int trans, int64_t n, int64_t ncols,
                   const float* X, int64_t ldx, float* Y, int64_t ldy, void* xs_work,
                   uint8_t* flags, int* err, cudaStream_t st) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc::encode_fn();
  if (!enc || !gemm_tc_supported(A, lda, n)) return 1;
  const int64_t kpad = ((n + TK - 1) / TK) * TK;
  const int nct = (int)((ncols + TN - 1) / TN);
  const int nkt = (int)(kpad / TK);
  __nv_bfloat16* Xs = (__nv_bfloat16*)xs_work;
  // A: FP32, dims (columns, rows), row stride lda; the box is one raw stage
  CUtensorMap tmA, tmX;
  const cuuint64_t adim[2] = {(cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t astr[1] = {(cuuint64_t)lda * 4};
  const cuuint32_t abox[2] = {trans ? (cuuint32_t)TM : (cuuint32_t)TK,
                              trans ? (cuuint32_t)TK : (cuuint32_t)TM};
  const cuuint32_t one[2] = {1, 1};
  if (enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)A, adim, astr, abox, one,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 2;
  // split X: BF16, dims (kpad, 3 * 64 * nct), 64 x 64 boxes with the 128-byte swizzle
  const cuuint64_t xdim[2] = {(cuuint64_t)kpad, (cuuint64_t)3 * TN * nct};
  const cuuint64_t xstr[1] = {(cuuint64_t)kpad * 2};
  const cuuint32_t xbox[2] = {(cuuint32_t)TK, (cuuint32_t)TN};
  if (enc(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)Xs, xdim, xstr, xbox, one,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 2;
  count_launches(2);
  k_split_x<<<dim3(nkt, nct), 256, 0, st>>>(X, ldx, n, ncols, kpad, nct, Xs, flags);
  const size_t smem = gemm_tc_smem_bytes();
  static std::atomic<uint32_t> done[2] = {{0}, {0}};
  // column tiles of one row block run side by side, so A is read from HBM once
  dim3 grid((unsigned)nct, (unsigned)((n + TM - 1) / TM));
  if (trans) {
    raise_smem_limit((const void*)k_gemm_tc<1>, done[1]);
    k_gemm_tc<1><<<grid, NTHREADS, smem, st>>>(tmA, tmX, n, ncols, flags, Y, ldy, err, wait_limit());
  } else {
    raise_smem_limit((const void*)k_gemm_tc<0>, done[0]);
    k_gemm_tc<0><<<grid, NTHREADS, smem, st>>>(tmA, tmX, n, ncols, flags, Y, ldy, err, wait_limit());
  }
  return 0;
}

}  // namespace hm
