// Sampling GEMM of the FP32 dense operator with FP64 samples (HM_A32) on the
// 5th-generation tensor cores: Y = op(A) X, A FP32, X and Y FP64, to about
// 2^-40 relative accuracy per product term (the FP64 black-box products
// A Omega / A^* Omega of the compression figures, without FP64 arithmetic in
// the contraction).
//
// Exact-accumulation split: inside one 64-wide K tile every row of op(A) and
// every column of X is scaled by a power of two so that its largest entry lies
// in [64, 128), and cut into four 8-bit integer slices (a = sum_s a_s 2^(-8(s-1))
// up to the scale, |a_s| <= 128, each exact in BF16).  A BF16 x BF16 product of
// slices is an integer below 2^14, and the products of one order d = s + t
// (d = 2..5, the terms of relative weight >= 2^-24) summed over the tile stay
// below 2^24, so the FP32 accumulators in TMEM hold them EXACTLY whatever the
// tensor cores' rounding.  Orders above 5 (relative weight <= 2^-32) are not
// formed.  Per tile and output element the drain adds
//     2^(e_A + e_X - 14) (L + 2^-8 M + 2^-16 C + 2^-24 D)
// (L, M, C, D: the exact sums of orders 2..5) into an FP32 double-float
// (hi, lo): the leading term through an error-free TwoSum, the smaller ones
// into lo.  Y = hi + lo in FP64.
//
// Block: 128 rows of op(A) x 64 columns of X, eighteen warps:
//   warp 17 (one lane): TMA loads of the FP32 tile of A into one raw stage;
//   warps 0-7: move the raw tile to registers (releasing the stage), find the
//     row scales, cut the slices into two operand stages (K-major, 128-byte
//     swizzle); one lane loads the pre-cut X slices by TMA;
//   warp 8: allocates 512 TMEM columns; one lane issues the MMAs (up to ten
//     products per 16-wide K step) into the four order accumulators;
//   warps 9-16: drain (two warps per TMEM lane quarter, 32 columns each) and
//     write Y.
// All-zero K tiles of X are skipped.  Every mbarrier wait is bounded; on
// timeout the block raises the error flag, writes NaN, lets its own TMA copies
// land and leaves; TMEM is released unless the wait for its MMAs timed out.
#include "tc_util.cuh"

namespace hm {
namespace {

using namespace tc;

constexpr int TM = 128, TN = 64, TK = 64;
constexpr int NSL = 4;                  // slices of A and of X
constexpr int A_SLICE = TM * TK * 2;    // 16 KB
constexpr int B_SLICE = TN * TK * 2;    // 8 KB
constexpr int RAW_BYTES = TM * TK * 4;  // 32 KB
constexpr int STAGE_BYTES = NSL * A_SLICE + NSL * B_SLICE;  // 96 KB
constexpr int SSTAGES = 2;
constexpr int LAYOUT_BYTES = RAW_BYTES + SSTAGES * STAGE_BYTES;  // 224 KB
constexpr int NCONV = 256, NDRAIN = 256, NTHREADS = 576;
constexpr int W_MMA = 8, W_DRAIN0 = 9, W_TMA = 17;
constexpr uint32_t TMEM_COLS = 512;  // 2 buffers x 4 orders x 64 columns
constexpr int EXP_BIAS = 127;        // row exponents stored as uint8 e + 127, e in [-120, 128]

__device__ __forceinline__ float pow2f(int k) {  // 2^k for k in [-126, 127]
  return __int_as_float((k + 127) << 23);
}

// exponent e with |x| < 2^e for x = the largest magnitude (0 for x == 0)
__device__ __forceinline__ int exp_above(float x) {
  if (!(x > 0.f)) return 0;
  int e;
  frexpf(x, &e);
  return e;
}

// Cut v (|v| < 128, a multiple of 2^-24 of the scale) into four 8-bit integers.
__device__ __forceinline__ void cut4(float v, float& s1, float& s2, float& s3, float& s4) {
  s1 = rintf(v);
  float r = (v - s1) * 256.f;
  s2 = rintf(r);
  r = (r - s2) * 256.f;
  s3 = rintf(r);
  r = (r - s3) * 256.f;
  s4 = rintf(r);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// X (FP64, column-major n x ncols) -> per (K tile, column) exponents and four
// BF16 integer slices, layout Xs[((ct * 4 + t) * 64 + c) * kpad + k]; flags bit t
// set when slice t of the (kt, ct) tile has a nonzero entry.
__global__ __launch_bounds__(256) void k_split_x64(const double* __restrict__ X, int64_t ldx,
                                                   int64_t n, int64_t ncols, int64_t kpad,
                                                   int nct, __nv_bfloat16* __restrict__ Xs,
                                                   int* __restrict__ ex,
                                                   uint8_t* __restrict__ flags) {
  const int kt = blockIdx.x, ct = blockIdx.y;
  const int tid = threadIdx.x;
  const int c = tid >> 2, kq = tid & 3;  // column c, 16 rows k = kq*16 .. kq*16+15
  const int64_t col = (int64_t)ct * TN + c;
  __shared__ int fl;
  if (tid == 0) fl = 0;
  double v[16];
  double mx = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int64_t row = (int64_t)kt * TK + kq * 16 + i;
    v[i] = (row < n && col < ncols) ? X[row + col * ldx] : 0.0;
    mx = fmax(mx, fabs(v[i]));
  }
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  __syncthreads();
  int bits = 0;
  const int64_t base = (int64_t)ct * NSL * TN;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int64_t row = (int64_t)kt * TK + kq * 16 + i;
    double r = ldexp(v[i], 7 - e);
    double s[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      s[t] = rint(r);
      r = (r - s[t]) * 256.0;
      bits |= (s[t] != 0.0) ? (1 << t) : 0;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
      Xs[(base + t * TN + c) * kpad + row] = __float2bfloat16_rn((float)s[t]);
  }
  if (bits) atomicOr(&fl, bits);
  if (kq == 0) ex[((int64_t)kt * nct + ct) * TN + c] = e;
  __syncthreads();
  if (tid == 0) flags[(int64_t)kt * nct + ct] = (uint8_t)fl;
}

// instruction order of the products: every accumulator's first MMA (t = 1)
// comes first, so that it overwrites
__constant__ int8_t kProdS[10] = {1, 2, 3, 4, 1, 2, 3, 1, 2, 1};
__constant__ int8_t kProdT[10] = {1, 1, 1, 1, 2, 2, 2, 3, 3, 4};

template <int TRANS>
__global__ __launch_bounds__(NTHREADS, 1) void k_gemm_esg(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX, int64_t n,
    int64_t ncols, const uint8_t* __restrict__ flags, const int* __restrict__ ex,
    double* __restrict__ Y, int64_t ldy, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t raw_full, raw_empty, st_full[SSTAGES], x_full[SSTAGES],
      st_empty[SSTAGES], acc_full[2], acc_empty[2], bar_final, exp_ready[4];
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;
  // row exponents (+127) of the last four tiles; exp_ready[i] completes a phase
  // when the cutters have written entry i (the drain reads it four tiles later
  // at the latest, so a ring of four never overtakes it)
  __shared__ uint8_t expa[4][TM];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ct = blockIdx.x, mt = blockIdx.y, nct = gridDim.x;
  const int64_t m0 = (int64_t)mt * TM;
  const int nkt = (int)((n + TK - 1) / TK);
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sbase = smem_raw + (base - raw);
  const uint32_t raw_addr = base, stage_addr0 = base + RAW_BYTES;

  if (tid == 0) {
    abort_flag = 0;
    mbar_init(smem_u32(&raw_full), 1);
    mbar_init(smem_u32(&raw_empty), NCONV);
    for (int i = 0; i < SSTAGES; ++i) {
      mbar_init(smem_u32(&st_full[i]), NCONV);
      mbar_init(smem_u32(&x_full[i]), 1);
      mbar_init(smem_u32(&st_empty[i]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), NDRAIN);
    }
    mbar_init(smem_u32(&bar_final), 1);
    for (int i = 0; i < 4; ++i) mbar_init(smem_u32(&exp_ready[i]), NCONV);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == W_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;
  auto active = [&](int kt) -> int { return flags[(int64_t)kt * nct + ct]; };

  if (warp == W_TMA) {
    // ---------------------------------------------------------- TMA of A
    if (lane == 0) {
      int it = 0;
      for (int kt = 0; kt < nkt; ++kt) {
        if (!active(kt)) continue;
        if (!mbar_wait(smem_u32(&raw_empty), (it & 1) ^ 1, &abort_flag)) break;
        mbar_arrive_tx(smem_u32(&raw_full), RAW_BYTES);
        if (!TRANS)
          tma_load_2d(raw_addr, &tmA, kt * TK, (int)m0, smem_u32(&raw_full));
        else
          tma_load_2d(raw_addr, &tmA, (int)m0, kt * TK, smem_u32(&raw_full));
        ++it;
      }
      if (it > 0) mbar_wait_drain(smem_u32(&raw_full), (it - 1) & 1);
    }
  } else if (warp < 8) {
    // ---------------------------------------------------------- cut A, TMA of X
    int it = 0, xissued = 0;
    for (int kt = 0; kt < nkt && !abort_flag; ++kt) {
      const int fl = active(kt);
      if (!fl) continue;
      const int s = it % SSTAGES;
      if (!mbar_wait(smem_u32(&st_empty[s]), ((it / SSTAGES) & 1) ^ 1, &abort_flag)) break;
      const uint32_t st = stage_addr0 + (uint32_t)s * STAGE_BYTES;
      if (tid == 0) {
        mbar_arrive_tx(smem_u32(&x_full[s]), (uint32_t)__popc(fl & 15) * B_SLICE);
        for (int t = 0; t < NSL; ++t)
          if (fl & (1 << t))
            tma_load_2d(st + NSL * A_SLICE + t * B_SLICE, &tmX, kt * TK, (ct * NSL + t) * TN,
                        smem_u32(&x_full[s]));
        xissued = it + 1;
      }
      if (!mbar_wait(smem_u32(&raw_full), it & 1, &abort_flag)) break;
      const unsigned char* rw = sbase;  // the raw stage sits at the aligned base
      unsigned char* sp = sbase + (st - base);
      uint8_t* ea = expa[it & 3];
      if (!TRANS) {
        // raw [128 rows][64 k]; pass p: rows 16p .. 16p+15, 16 threads per row
        float4 v[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const int f = p * NCONV + tid, m = f >> 4, k4 = f & 15;
          v[p] = *reinterpret_cast<const float4*>(rw + m * 256 + k4 * 16);
        }
        mbar_arrive(smem_u32(&raw_empty));  // the raw stage is free for the next tile
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const int f = p * NCONV + tid, m = f >> 4, k4 = f & 15;
          float mx = fmaxf(fmaxf(fabsf(v[p].x), fabsf(v[p].y)), fmaxf(fabsf(v[p].z), fabsf(v[p].w)));
#pragma unroll
          for (int o = 1; o < 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          const int e = max(exp_above(mx), -120);
          if (k4 == 0) ea[m] = (uint8_t)(e + EXP_BIAS);
          const float sc = pow2f(7 - e);
          float a[4] = {v[p].x * sc, v[p].y * sc, v[p].z * sc, v[p].w * sc};
          float sl[4][4];
#pragma unroll
          for (int i = 0; i < 4; ++i) cut4(a[i], sl[0][i], sl[1][i], sl[2][i], sl[3][i]);
          const uint32_t off = sw_off(m, k4 >> 1) + (uint32_t)((k4 & 1) * 8);
#pragma unroll
          for (int t = 0; t < NSL; ++t)
            *reinterpret_cast<uint2*>(sp + t * A_SLICE + off) =
                make_uint2(pack_bf16(sl[t][0], sl[t][1]), pack_bf16(sl[t][2], sl[t][3]));
        }
      } else {
        // raw [64 k][128 m]; thread (m, half) takes k = 32 half .. 32 half + 31
        const int m = tid & (TM - 1), h = tid >> 7;
        // partial row maxima live in the last KB of this stage's slice 3 until the
        // slices are written
        float* pmax = reinterpret_cast<float*>(sp + 3 * A_SLICE + A_SLICE - 2 * TM * 4);
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i)
          v[i] = *reinterpret_cast<const float*>(rw + ((h * 32 + i) * TM + m) * 4);
        mbar_arrive(smem_u32(&raw_empty));
        float mx = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) mx = fmaxf(mx, fabsf(v[i]));
        pmax[h * TM + m] = mx;
        asm volatile("bar.sync 1, 256;" ::: "memory");
        const float rmx = fmaxf(pmax[m], pmax[TM + m]);
        asm volatile("bar.sync 1, 256;" ::: "memory");  // read before the slices overwrite it
        const int e = max(exp_above(rmx), -120);
        if (h == 0) ea[m] = (uint8_t)(e + EXP_BIAS);
        const float sc = pow2f(7 - e);
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // 16-byte chunk q of this half: k = 32 h + 8 q ..
          float sl[4][8];
#pragma unroll
          for (int i = 0; i < 8; ++i)
            cut4(v[q * 8 + i] * sc, sl[0][i], sl[1][i], sl[2][i], sl[3][i]);
          const uint32_t off = sw_off(m, h * 4 + q);
#pragma unroll
          for (int t = 0; t < NSL; ++t)
            *reinterpret_cast<uint4*>(sp + t * A_SLICE + off) =
                make_uint4(pack_bf16(sl[t][0], sl[t][1]), pack_bf16(sl[t][2], sl[t][3]),
                           pack_bf16(sl[t][4], sl[t][5]), pack_bf16(sl[t][6], sl[t][7]));
        }
      }
      mbar_arrive(smem_u32(&exp_ready[it & 3]));
      fence_proxy_async();
      mbar_arrive(smem_u32(&st_full[s]));
      ++it;
    }
    if (tid == 0)
      for (int j = (xissued > SSTAGES ? xissued - SSTAGES : 0); j < xissued; ++j)
        mbar_wait_drain(smem_u32(&x_full[j % SSTAGES]), (j / SSTAGES) & 1);
  } else if (warp == W_MMA) {
    // ---------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32();
      int it = 0;
      bool ok = true;
      for (int kt = 0; kt < nkt && ok; ++kt) {
        const int fl = active(kt);
        if (!fl) continue;
        const int b = it & 1, s = it % SSTAGES;
        ok = mbar_wait(smem_u32(&acc_empty[b]), ((it >> 1) & 1) ^ 1, &abort_flag) &&
             mbar_wait(smem_u32(&st_full[s]), (it / SSTAGES) & 1, &abort_flag) &&
             mbar_wait(smem_u32(&x_full[s]), (it / SSTAGES) & 1, &abort_flag);
        if (!ok) break;
        tc_fence_after();
        const uint32_t st = stage_addr0 + (uint32_t)s * STAGE_BYTES;
        const uint32_t dbase = tmem + (uint32_t)(b * 4 * TN);
        uint32_t started = 0;  // bit d: accumulator of order d + 2 already written
#pragma unroll
        for (int kk = 0; kk < TK / 16; ++kk) {
#pragma unroll
          for (int p = 0; p < 10; ++p) {
            const int sa = kProdS[p] - 1, sb = kProdT[p] - 1, d = sa + sb;
            if (!(fl & (1 << sb))) continue;
            const uint64_t ad = sw128_desc(st + sa * A_SLICE + kk * 32);
            const uint64_t bd = sw128_desc(st + NSL * A_SLICE + sb * B_SLICE + kk * 32);
            mma_bf16(dbase + (uint32_t)(d * TN), ad, bd, idesc, (started >> d) & 1u);
            started |= 1u << d;
          }
        }
        mma_commit(smem_u32(&st_empty[s]));
        mma_commit(smem_u32(&acc_full[b]));
        ++it;
      }
      mma_commit(smem_u32(&bar_final));
      if (!mbar_wait(smem_u32(&bar_final), 0, &abort_flag)) abort_flag = 2;
    }
  } else {
    // ---------------------------------------------------------- drain / epilogue
    const int dw = warp - W_DRAIN0;  // 0..7
    const int q4 = warp & 3;         // TMEM lane quarter
    const int half = dw >> 2;        // columns 32 half .. 32 half + 31
    const int r = q4 * 32 + lane;
    float hi[32], lo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
    const int64_t colbase = (int64_t)ct * TN + half * 32;
    int it = 0;
    for (int kt = 0; kt < nkt; ++kt) {
      const int fl = active(kt);
      if (!fl) continue;
      const int b = it & 1;
      const int exl = ex[((int64_t)kt * nct + ct) * TN + half * 32 + lane];  // column lane
      if (!mbar_wait(smem_u32(&acc_full[b]), (it >> 1) & 1, &abort_flag)) break;
      if (!mbar_wait(smem_u32(&exp_ready[it & 3]), (it >> 2) & 1, &abort_flag)) break;
      tc_fence_after();
      const int ea = (int)expa[it & 3][r] - EXP_BIAS;
      const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * 4 * TN + half * 32);
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        float sc[16], v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int e = ea + __shfl_sync(0xffffffffu, exl, g * 16 + j) - 14;
          sc[j] = (e >= -126 && e <= 127) ? pow2f(e) : ldexpf(1.f, e);
        }
        // order 2: exact integer sums, added through TwoSum
        tmem_ld16(tl + 0 * TN + g * 16, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int jj = g * 16 + j;
          const float t = v[j] * sc[j];
          const float sum = hi[jj] + t;
          const float bp = sum - hi[jj];
          lo[jj] += (hi[jj] - (sum - bp)) + (t - bp);
          hi[jj] = sum;
        }
        // orders 3..5: 2^-8, 2^-16 and 2^-24 of the leading term, into lo
        tmem_ld16(tl + 1 * TN + g * 16, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) lo[g * 16 + j] = fmaf(v[j], sc[j] * 0.00390625f, lo[g * 16 + j]);
        tmem_ld16(tl + 2 * TN + g * 16, v);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          lo[g * 16 + j] = fmaf(v[j], sc[j] * 1.52587890625e-05f, lo[g * 16 + j]);
        tmem_ld16(tl + 3 * TN + g * 16, v);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          lo[g * 16 + j] = fmaf(v[j], sc[j] * 5.9604644775390625e-08f, lo[g * 16 + j]);
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&acc_empty[b]));
      ++it;
    }
    const int64_t grow = m0 + r;
    const bool bad = abort_flag != 0;
    if (grow < n) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int64_t col = colbase + j;
        if (col < ncols)
          Y[grow + col * ldy] = bad ? __longlong_as_double(0x7ff8000000000000ll)
                                    : (double)hi[j] + (double)lo[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (abort_flag && tid == 0) atomicExch(err, 1);
  if (warp == W_MMA && abort_flag != 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

}  // namespace

size_t gemm_esg_smem_bytes() { return (size_t)LAYOUT_BYTES + 1024; }

// bytes of the pre-cut X workspace: four BF16 slices per padded column tile,
// then one int exponent per (K tile, column)
int64_t gemm_esg_work_bytes(int64_t n, int64_t ncols) {
  const int64_t kpad = ((n + TK - 1) / TK) * TK;
  const int64_t nct = (ncols + TN - 1) / TN;
  const int64_t xs = nct * NSL * TN * kpad * 2;
  return ((xs + 255) / 256) * 256 + (kpad / TK) * nct * TN * 4;
}

int launch_gemm_esg(const float* A, int64_t lda, int trans, int64_t n, int64_t ncols,
                    const double* X, int64_t ldx, double* Y, int64_t ldy, void* work,
                    uint8_t* flags, int* err, cudaStream_t st) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc::encode_fn();
  if (!enc || !gemm_tc_supported(A, lda, n)) return 1;
  const int64_t kpad = ((n + TK - 1) / TK) * TK;
  const int nct = (int)((ncols + TN - 1) / TN);
  const int nkt = (int)(kpad / TK);
  __nv_bfloat16* Xs = (__nv_bfloat16*)work;
  const int64_t xs_bytes = (int64_t)nct * NSL * TN * kpad * 2;
  int* ex = (int*)((unsigned char*)work + ((xs_bytes + 255) / 256) * 256);
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
  const cuuint64_t xdim[2] = {(cuuint64_t)kpad, (cuuint64_t)NSL * TN * nct};
  const cuuint64_t xstr[1] = {(cuuint64_t)kpad * 2};
  const cuuint32_t xbox[2] = {(cuuint32_t)TK, (cuuint32_t)TN};
  if (enc(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)Xs, xdim, xstr, xbox, one,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 2;
  count_launches(2);
  k_split_x64<<<dim3(nkt, nct), 256, 0, st>>>(X, ldx, n, ncols, kpad, nct, Xs, ex, flags);
  const size_t smem = gemm_esg_smem_bytes();
  static bool configured[2] = {false, false};
  dim3 grid((unsigned)nct, (unsigned)((n + TM - 1) / TM));
  if (trans) {
    if (!configured[1])
      cudaFuncSetAttribute(k_gemm_esg<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured[1] = true;
    k_gemm_esg<1><<<grid, NTHREADS, smem, st>>>(tmA, tmX, n, ncols, flags, ex, Y, ldy, err);
  } else {
    if (!configured[0])
      cudaFuncSetAttribute(k_gemm_esg<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured[0] = true;
    k_gemm_esg<0><<<grid, NTHREADS, smem, st>>>(tmA, tmX, n, ncols, flags, ex, Y, ldy, err);
  }
  return 0;
}

}  // namespace hm
