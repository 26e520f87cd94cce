// Sampling GEMM of the FP32 dense operator with FP64 samples (HM_A32) on the
// 5th-generation tensor cores: Y = op(A) X, A FP32, X and Y FP64, to about
// 2^-32 of (max slice)^2 relative per product term (the FP64 black-box products
// A Omega / A^* Omega of the compression figures, without FP64 arithmetic in
// the contraction).
//
// Exact-accumulation split: every row of op(A) and every column of X inside a
// window of 256 K values (the A exponents are recorded once per operator) is
// scaled by a power of two so that its largest entry lies in [64, 128), and cut
// into four 8-bit integer slices
// (a = sum_s a_s 2^(-8(s-1)) up to the scale, |a_s| <= 128, each exact in BF16).
// A BF16 x BF16 product of slices is an integer of magnitude <= 2^14, and the
// products of one order d = s + t (d = 2..5, at most four of them) summed over
// a window of 256 K values stay within 2^24, so the FP32 accumulators in TMEM
// hold them EXACTLY whatever the tensor cores' rounding.  Orders above 5 are
// not formed.  Per window and output element the drain adds
//     2^(e_A + e_X - 14) (L + 2^-8 M + 2^-16 C + 2^-24 D)
// (L, M, C, D: the exact sums of orders 2..5) into an FP32 double-float
// (hi, lo), every term through an error-free TwoSum.  Y = hi + lo in FP64.
//
// MMA form: one chain of same-shape MMAs per K tile.  A stage holds the four A
// slices and the X slices stacked as seven 64-row blocks [0 0 0 x1 x2 x3 x4]
// (three zero blocks written once).  A slice s times the 256 rows starting at
// block 4 - s is [0 ... x1 .. x(5-s)], so its N = 256 product lands, column
// block j, in the accumulator of order j + 2 for every s: all sixteen MMAs of
// a 32-wide K tile (4 slices x 2 K steps) have the same accumulator and shape
// and are ordered by the tensor pipe without waits.  The zero blocks cost 6 of
// 16 products' worth of tensor work; the MMAs are large enough (128 x 256 x 16)
// that one thread's issue keeps the pipe fed.
//
// Block: 128 rows of op(A) x 64 columns of X, eighteen warps:
//   warp 17 (one lane): TMA loads of the FP32 tiles of A (128 x 32) into four
//     raw stages;
//   warps 0-7: move a raw tile to registers (releasing the stage), scale and
//     cut the slices into one of two operand stages (K-major, 64-byte swizzle);
//     one lane loads the pre-cut X slices by TMA.  An entry that does not fit
//     its recorded row scale (the operator changed after the scales were taken)
//     aborts the block, whose outputs are then NaN;
//   warp 8: allocates 512 TMEM columns (two windows x four orders x 64
//     columns); one lane issues the MMAs;
//   warps 9-16: drain once per window (two warps per TMEM lane quarter, 32
//     columns each) and write Y.
// All-zero K tiles of X are skipped; the four X slices of an active tile are
// always loaded (a zero slice contributes zeros).  Every mbarrier wait is bounded
// (the pipeline waits by the limit the host sets, hm_set_wait_limit); on timeout
// the block raises the error flag, writes NaN, lets its own TMA copies land and
// its issued MMAs complete (waits of the full limit) and leaves; TMEM is
// released unless even the full-limit wait for its MMAs ran out.
#include <algorithm>
#include <cstring>
#include <atomic>

#include "tc_util.cuh"

namespace hm {
namespace {

using namespace tc;

constexpr int TM = 128, TN = 64, TK = 32;  // TK: the K extent of a stage
constexpr int NSL = 4;                  // slices of A and of X
constexpr int A_SLICE = TM * TK * 2;    // 8 KB: 128 rows x 64 bytes
constexpr int XB = TN * TK * 2;         // 4 KB: one X slice, 64 rows x 64 bytes
constexpr int XZ = 3;                   // zero blocks before x1
constexpr int X_BYTES = (XZ + NSL) * XB;                 // 28 KB
constexpr int STAGE_BYTES = NSL * A_SLICE + X_BYTES;     // 60 KB
constexpr int SSTAGES = 3;
constexpr int RAW_BYTES = TM * TK * 4;  // 16 KB
constexpr int RSTAGES = 2;
constexpr int RAW_REGION = RSTAGES * RAW_BYTES;          // 32 KB
constexpr int LAYOUT_BYTES = RAW_REGION + SSTAGES * STAGE_BYTES;  // 212 KB
constexpr int NCONV = 256, NDRAIN = 256, NTHREADS = 608;
constexpr int W_MMA = 8, W_DRAIN0 = 9, W_TMA = 17, W_XTMA = 18;
constexpr uint32_t TMEM_COLS = 512;  // 2 buffers x 4 orders x 64 columns
constexpr int WIN_ROWS = 256;        // K values per exact accumulation window
constexpr int WIN_TILES = WIN_ROWS / TK;
constexpr int KPAD = 64;             // K padding of the pre-cut X (k_split_x64's rows)
constexpr int MAX_KT = 16384;        // K tiles a call may have (n <= 524288)

static_assert(STAGE_BYTES % 1024 == 0 && RAW_BYTES % 1024 == 0, "1 KB aligned stages");

// Shared-memory matrix descriptor: K-major, 64-byte swizzle (16-byte chunk c of
// row r at chunk c ^ ((r >> 1) & 3)), 8-row groups 512 bytes apart; start
// address and offsets in 16-byte units.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;   // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)4 << 61;            // 64-byte swizzle
  return d;
}
// byte offset of 16-byte chunk q (0..3) of row m in a 64-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t sw64_off(int m, int q) {
  return (uint32_t)((m >> 3) * 512 + (m & 7) * 64 + ((q ^ ((m >> 1) & 3)) << 4));
}

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

// Round to the nearest integer, ties to even, for |x| < 2^22: adding 1.5 * 2^23
// lands in [2^23, 2^24), where the FP32 spacing is 1, so the add rounds x and
// the subtraction is exact.  Two adds on the FMA pipe instead of one rounding
// instruction on the slower conversion pipe; the compiler does not reassociate
// the pair (no fast-math).
__device__ __forceinline__ float round_int(float x) {
  return (x + 12582912.f) - 12582912.f;
}

// Cut v (|v| < 128, a multiple of 2^-24 of the scale) into four 8-bit integers
// (the digits of v rounded to a multiple of 2^-24, each in [-128, 128]).
__device__ __forceinline__ void cut4(float v, float& s1, float& s2, float& s3, float& s4) {
  s1 = round_int(v);
  float r = (v - s1) * 256.f;
  s2 = round_int(r);
  r = (r - s2) * 256.f;
  s3 = round_int(r);
  r = (r - s3) * 256.f;
  s4 = round_int(r);
}

// Two digits as a BF16 pair (lo in the low half).  A digit is an integer of at
// most 8 significant bits, so its FP32 pattern ends in 16 zero bits and its BF16
// pattern is the FP32 pattern's upper half: one byte permute, no rounding.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// Exponents of A per row and window of 256 columns: e_row[i * nw + w] = e with
// max over the window of |A(i, j)| < 2^e (clamped to >= -120).  One warp per
// row, eight entries per lane and window.
__global__ __launch_bounds__(256) void k_row_exp(const float* __restrict__ A, int64_t lda,
                                                 int64_t n, int nw, int* __restrict__ e_row) {
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* a = A + row * lda;
  for (int w = 0; w < nw; ++w) {
    float mx = 0.f;
    for (int64_t j = (int64_t)w * WIN_ROWS + lane; j < n && j < (int64_t)(w + 1) * WIN_ROWS;
         j += 32)
      mx = fmaxf(mx, fabsf(a[j]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) e_row[row * nw + w] = max(exp_above(mx), -120);
  }
}

// The same per column and window of 256 rows (the rows of op(A) = A^T): one
// thread per column, rows streamed.
__global__ __launch_bounds__(256) void k_col_exp(const float* __restrict__ A, int64_t lda,
                                                 int64_t n, int nw, int* __restrict__ e_col) {
  const int64_t col = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (col >= n) return;
  for (int w = 0; w < nw; ++w) {
    float mx = 0.f;
    const int64_t i1 = (n < (int64_t)(w + 1) * WIN_ROWS) ? n : (int64_t)(w + 1) * WIN_ROWS;
#pragma unroll 8
    for (int64_t i = (int64_t)w * WIN_ROWS; i < i1; ++i) mx = fmaxf(mx, fabsf(A[i * lda + col]));
    e_col[col * nw + w] = max(exp_above(mx), -120);
  }
}

// X (FP64, column-major n x ncols) -> per (window, column) exponents and four
// BF16 integer slices, laid out as the GEMM's shared memory wants them: per
// (column tile ct, K tile kt) one contiguous 16 KB block of 256 rows
// (row t * 64 + c: slice t of column c) x 32 K values, each row's four 16-byte
// chunks in 64-byte-swizzle order, so one 1-D bulk copy lands a tile in place.
// Flags of (kt, ct) nonzero when that K tile has a nonzero slice.  Block: one
// window (256 rows) x 64 columns; thread (c, q) covers rows 64 q .. 64 q + 63
// of the window (kpad is a multiple of 64).
__global__ __launch_bounds__(256) void k_split_x64(const double* __restrict__ X, int64_t ldx,
                                                   int64_t n, int64_t ncols, int64_t kpad,
                                                   int nct, __nv_bfloat16* __restrict__ Xs,
                                                   int* __restrict__ ex,
                                                   uint8_t* __restrict__ flags) {
  constexpr int QR = WIN_ROWS / 4;  // rows per thread
  const int win = blockIdx.x, ct = blockIdx.y;
  const int tid = threadIdx.x;
  const int c = tid >> 2, q = tid & 3;
  const int64_t col = (int64_t)ct * TN + c;
  const int64_t r0 = (int64_t)win * WIN_ROWS + q * QR;
  __shared__ int fl[WIN_TILES];
  if (tid < WIN_TILES) fl[tid] = 0;
  double mx = 0.0;
  for (int i = 0; i < QR; ++i) {
    const int64_t row = r0 + i;
    if (row < n && col < ncols) mx = fmax(mx, fabs(X[row + col * ldx]));
  }
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  __syncthreads();
  int bits[QR / TK] = {};
  if (r0 < kpad) {
    for (int i = 0; i < QR; ++i) {
      const int64_t row = r0 + i;
      double r = (row < n && col < ncols) ? ldexp(X[row + col * ldx], 7 - e) : 0.0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const double st = rint(r);
        r = (r - st) * 256.0;
        bits[i / TK] |= (st != 0.0) ? (1 << t) : 0;
        const int rr = t * TN + c, kk = (int)(row % TK);
        const int64_t tile = (int64_t)ct * (kpad / TK) + row / TK;
        Xs[(tile * (NSL * TN) + rr) * TK + ((((kk >> 3) ^ ((rr >> 1) & 3))) << 3) + (kk & 7)] =
            __float2bfloat16_rn((float)st);
      }
    }
  }
#pragma unroll
  for (int h = 0; h < QR / TK; ++h)
    if (bits[h]) atomicOr(&fl[q * (QR / TK) + h], bits[h]);
  if (q == 0) ex[((int64_t)win * nct + ct) * TN + c] = e;
  __syncthreads();
  if (tid < WIN_TILES) {
    const int64_t kt = (int64_t)win * WIN_TILES + tid;
    if (kt * TK < kpad) flags[kt * nct + ct] = (uint8_t)fl[tid];
  }
}

// Named barrier 1 of the 256 cutter threads (warps 0-7), and its AND-reduction
// form: the generating cutters (GEN) stage table windows in shared memory and
// must leave their loop together.
__device__ __forceinline__ void cutters_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ bool cutters_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// GEN = 1: the operator is the matrix-free log kernel of the ellipse (see
// launch_gemm_esg_gen): the cutters generate each tile's entries from two
// tables instead of reading a TMA tile of A (no A bytes from HBM); the
// operator is symmetric, so only TRANS = 0 is instantiated.
template <int TRANS, int GEN>
__global__ __launch_bounds__(NTHREADS, 1) void k_gemm_esg(
    const __grid_constant__ CUtensorMap tmA, const __nv_bfloat16* __restrict__ Xs, int64_t n,
    int64_t ncols, const uint8_t* __restrict__ flags, const int* __restrict__ ex,
    const int* __restrict__ e_rows, double* __restrict__ Y, int64_t ldy, int* __restrict__ err,
    long long poll_limit, const float* __restrict__ tabS, const float* __restrict__ tabP) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t raw_full[RSTAGES], raw_empty[RSTAGES], st_full[SSTAGES],
      x_full[SSTAGES], st_empty[SSTAGES], acc_full[2], acc_empty[2], bar_final;
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;
  __shared__ int win_lo, win_hi;  // this block's share of the windows (split over K)
  __shared__ uint32_t act_bits[MAX_KT / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ct = blockIdx.x, mt = blockIdx.y, nct = gridDim.x;
  const int64_t m0 = (int64_t)mt * TM;
  const int nkt = (int)((n + TK - 1) / TK);
  const int nwin = (nkt + WIN_TILES - 1) / WIN_TILES;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sbase = smem_raw + (base - raw);
  const uint32_t raw_addr = base, stage_addr0 = base + RAW_REGION;
  // 2^(7 - e), e the exponent of row m of this block in window w (1 past n)
  auto row_scale = [&](int m, int w) -> float {
    return pow2f(7 - ((m0 + m < n) ? e_rows[(m0 + m) * nwin + w] : 0));
  };

  if (tid == 0) {
    abort_flag = 0;
    for (int i = 0; i < RSTAGES; ++i) {
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
      mbar_init(smem_u32(&acc_empty[b]), NDRAIN);
    }
    mbar_init(smem_u32(&bar_final), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the zero blocks in front of each stage's X slices, written once; the MMAs
  // read them through the async proxy
  for (int i = tid; i < SSTAGES * XZ * XB / 16; i += NTHREADS) {
    const int sidx = i / (XZ * XB / 16), o = i % (XZ * XB / 16);
    *reinterpret_cast<uint4*>(sbase + RAW_REGION + sidx * STAGE_BYTES + NSL * A_SLICE + o * 16) =
        make_uint4(0u, 0u, 0u, 0u);
  }
  fence_proxy_async();
  if (warp == W_TMA) {
    // blocks z = 0 .. gridDim.z - 1 of a row block share its active windows
    // (those with a nonzero K tile of X) in equal counts, in window order
    const int ks = (int)gridDim.z, z = (int)blockIdx.z;
    int lo = 0, hi = nwin;
    if (ks > 1) {
      auto win_active = [&](int w) -> bool {
        bool a = false;
        for (int t = 0; t < WIN_TILES; ++t) {
          const int kt = w * WIN_TILES + t;
          if (kt < nkt && flags[(int64_t)kt * nct + ct]) a = true;
        }
        return a;
      };
      int total = 0;
      for (int w0 = 0; w0 < nwin; w0 += 32) {
        const int w = w0 + lane;
        total += __popc(__ballot_sync(0xffffffffu, w < nwin && win_active(w)));
      }
      const int r0 = (int)((int64_t)z * total / ks), r1 = (int)((int64_t)(z + 1) * total / ks);
      int seen = 0, clo = nwin, chi = nwin;
      for (int w0 = 0; w0 < nwin; w0 += 32) {
        const int w = w0 + lane;
        const bool a = w < nwin && win_active(w);
        const unsigned b = __ballot_sync(0xffffffffu, a);
        const int rank = seen + __popc(b & ((1u << lane) - 1u));
        if (a && rank == r0) clo = w;
        if (a && rank == r1) chi = w;
        seen += __popc(b);
      }
      for (int o = 16; o > 0; o >>= 1) {
        clo = min(clo, __shfl_xor_sync(0xffffffffu, clo, o));
        chi = min(chi, __shfl_xor_sync(0xffffffffu, chi, o));
      }
      lo = clo;
      hi = (r1 >= total) ? nwin : chi;
    }
    if (lane == 0) { win_lo = lo; win_hi = hi; }
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
  const int wlo = win_lo, whi = win_hi;
  // one bit per K tile: nonzero X and inside this block's share of the windows
  // (every role walks the tiles; a shared-memory bit instead of a global load
  // per tile and role)
  for (int wd = tid; wd < (nkt + 31) / 32; wd += NTHREADS) {
    uint32_t b = 0;
    for (int i = 0; i < 32; ++i) {
      const int kt = wd * 32 + i, w = kt / WIN_TILES;
      if (kt < nkt && w >= wlo && w < whi && flags[(int64_t)kt * nct + ct]) b |= 1u << i;
    }
    act_bits[wd] = b;
  }
  __syncthreads();
  auto active = [&](int kt) -> int { return (act_bits[kt >> 5] >> (kt & 31)) & 1; };
  // the first active K tile at or after `from` (nkt if none)
  const int nwords = (nkt + 31) / 32;
  auto next_active = [&](int from) -> int {
    int wd = from >> 5;
    if (wd >= nwords) return nkt;
    uint32_t b = act_bits[wd] & (~0u << (from & 31));
    while (!b) {
      if (++wd >= nwords) return nkt;
      b = act_bits[wd];
    }
    return (wd << 5) + __ffs(b) - 1;
  };

  if (warp == W_TMA) {
    // ---------------------------------------------------------- TMA of A
    if (!GEN && lane == 0) {
      int it = 0;
      const uint64_t pol = l2_policy_evict_first();  // A is read once per call
      for (int kt = next_active(0); kt < nkt; kt = next_active(kt + 1)) {
        const int r = it % RSTAGES;
        if (!mbar_wait(smem_u32(&raw_empty[r]), ((it / RSTAGES) & 1) ^ 1, &abort_flag,
                       poll_limit))
          break;
        mbar_arrive_tx(smem_u32(&raw_full[r]), RAW_BYTES);
        if (!TRANS)
          tma_load_2d_hint(raw_addr + r * RAW_BYTES, &tmA, kt * TK, (int)m0,
                           smem_u32(&raw_full[r]), pol);
        else
          tma_load_2d_hint(raw_addr + r * RAW_BYTES, &tmA, (int)m0, kt * TK,
                           smem_u32(&raw_full[r]), pol);
        ++it;
      }
      // the copies in flight land before the block's shared memory is given up
      for (int j = (it > RSTAGES ? it - RSTAGES : 0); j < it; ++j)
        mbar_wait_drain(smem_u32(&raw_full[j % RSTAGES]), (j / RSTAGES) & 1);
    }
  } else if (GEN && warp < 8) {
    // ---------------------------------------------------------- generate A, cut, TMA of X
    // A(i, j) = (S[|i - j|] + P[i + j]) in float pairs: fl((Sh + Ph) + (Sl + Pl)),
    // 1 on the diagonal, 0 outside [0, n).  A tile's entries use TM + TK - 1
    // values of each table, staged in the (unused) raw region: window entry e
    // holds S[|d|] for i - j = d = m0 - k0 - (TK - 1) + e, and P[m0 + k0 + e].
    int it = 0;
    // Four shifted copies of each window (copy q holds window entry x + q at x),
    // so that every thread reads its four consecutive entries of a table as one
    // aligned float4: for row m the P entries start at m + 4 k4 and the S entries
    // (descending) at m - 4 k4 + TK - 4, both congruent to m mod 4.
    constexpr int WC = 164;  // floats per copy (16-byte multiple, covers index 161)
    float* win = reinterpret_cast<float*>(sbase);  // [table (Sh, Sl, Ph, Pl)][q][WC]
    // Thread e (< TM + TK - 1 <= NCONV) owns window entry e.  The next active
    // tile's entry is loaded from the (L2-resident) tables one tile ahead, so the
    // load latency hides behind the current tile's cut.
    float pv[4] = {0.f, 0.f, 0.f, 0.f};
    auto load_win = [&](int ktn) {
      pv[0] = pv[1] = pv[2] = pv[3] = 0.f;
      const int e = tid;
      if (e < TM + TK - 1) {
        const int64_t kn = (int64_t)ktn * TK;
        const int64_t d = m0 - kn - (TK - 1) + e, ad = d < 0 ? -d : d, sidx = m0 + kn + e;
        if (ad > 0 && ad < n) { pv[0] = tabS[ad]; pv[1] = tabS[n + ad]; }
        if (sidx < 2 * n - 1) { pv[2] = tabP[sidx]; pv[3] = tabP[2 * n - 1 + sidx]; }
      }
    };
    {
      const int k1 = next_active(0);
      if (k1 < nkt) load_win(k1);
    }
    constexpr int NP = TM * TK / 4 / NCONV;  // 4 passes: rows 32 p + tid / 8
    float scs[NP];                           // this thread's row scales in window scw
    int scw = -1;
    for (int kt = next_active(0); kt < nkt; kt = next_active(kt + 1)) {
      const int s = it % SSTAGES;
      const bool ok = !abort_flag &&
                      mbar_wait(smem_u32(&st_empty[s]), ((it / SSTAGES) & 1) ^ 1, &abort_flag,
                                poll_limit);
      // all cutters leave together (they share the table windows); the barrier
      // also orders the previous tile's window reads before the new writes
      if (!cutters_all(ok)) break;
      const uint32_t st = stage_addr0 + (uint32_t)s * STAGE_BYTES;
      const int64_t k0 = (int64_t)kt * TK;
      {
        const int e = tid;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int x = e - q;
          if (x >= 0 && x < WC)
#pragma unroll
            for (int a = 0; a < 4; ++a) win[(a * 4 + q) * WC + x] = pv[a];
        }
      }
      {
        const int k1 = next_active(kt + 1);
        if (k1 < nkt) load_win(k1);
      }
      cutters_sync();
      // tiles that hold a diagonal entry or reach past n take the per-entry fixes
      const bool fix = (m0 + TM > n) || (k0 + TK > n) || (m0 < k0 + TK && k0 < m0 + TM);
      const int dk = (int)(fix ? k0 - m0 : 0);  // i == j  <=>  m - (4 k4 + e) == dk
      const int mrow = (int)(n - m0 < TM ? n - m0 : TM), kcol = (int)(n - k0 < TK ? n - k0 : TK);
      unsigned char* sp = sbase + (st - base);
      int bad = 0;
      if (kt / WIN_TILES != scw) {
        scw = kt / WIN_TILES;
#pragma unroll
        for (int p = 0; p < NP; ++p) scs[p] = row_scale((p * NCONV + tid) >> 3, scw);
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const int f = p * NCONV + tid, m = f >> 3, k4 = f & 7;
        const float sc = scs[p];
        const int q = m & 3, ps = m + 4 * k4 - q, ds = m - 4 * k4 + (TK - 4) - q;
        const float4 sh4 = *reinterpret_cast<const float4*>(win + (0 * 4 + q) * WC + ds);
        const float4 sl4 = *reinterpret_cast<const float4*>(win + (1 * 4 + q) * WC + ds);
        const float4 ph4 = *reinterpret_cast<const float4*>(win + (2 * 4 + q) * WC + ps);
        const float4 pl4 = *reinterpret_cast<const float4*>(win + (3 * 4 + q) * WC + ps);
        // entry e: S at window index m - 4 k4 + TK - 1 - e (component 3 - e of the
        // S float4), P at m + 4 k4 + e (component e)
        const float shv[4] = {sh4.w, sh4.z, sh4.y, sh4.x}, slv[4] = {sl4.w, sl4.z, sl4.y, sl4.x};
        const float phv[4] = {ph4.x, ph4.y, ph4.z, ph4.w}, plv[4] = {pl4.x, pl4.y, pl4.z, pl4.w};
        float a[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float v = (shv[e] + phv[e]) + (slv[e] + plv[e]);
          if (fix) {
            const int kk = 4 * k4 + e;
            if (m - kk == dk) v = 1.f;
            if (m >= mrow || kk >= kcol) v = 0.f;
          }
          a[e] = v * sc;
        }
        float sl[4][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          bad |= !(fabsf(a[e]) < 128.f);
          cut4(a[e], sl[0][e], sl[1][e], sl[2][e], sl[3][e]);
        }
        const uint32_t off = sw64_off(m, k4 >> 1) + (uint32_t)((k4 & 1) * 8);
#pragma unroll
        for (int t = 0; t < NSL; ++t)
          *reinterpret_cast<uint2*>(sp + t * A_SLICE + off) =
              make_uint2(pack_bf16(sl[t][0], sl[t][1]), pack_bf16(sl[t][2], sl[t][3]));
      }
      if (bad) abort_flag = 3;
      fence_proxy_async();
      mbar_arrive(smem_u32(&st_full[s]));
      ++it;
    }
  } else if (warp < 8) {
    // ---------------------------------------------------------- cut A, TMA of X
    int it = 0;
    constexpr int NP = TM * TK / 4 / NCONV;  // 4 passes: rows 32 p + tid / 8 (not TRANS)
    float scs[NP];                           // this thread's row scales in window scw
    int scw = -1;
    for (int kt = next_active(0); kt < nkt && !abort_flag; kt = next_active(kt + 1)) {
      const int s = it % SSTAGES, r = it % RSTAGES;
      if (kt / WIN_TILES != scw) {  // (issued before the raw wait: the loads overlap it)
        scw = kt / WIN_TILES;
        if (!TRANS) {
#pragma unroll
          for (int p = 0; p < NP; ++p) scs[p] = row_scale((p * NCONV + tid) >> 3, scw);
        } else {
          scs[0] = row_scale(tid & (TM - 1), scw);
        }
      }
      if (!mbar_wait(smem_u32(&st_empty[s]), ((it / SSTAGES) & 1) ^ 1, &abort_flag, poll_limit))
        break;
      const uint32_t st = stage_addr0 + (uint32_t)s * STAGE_BYTES;
      if (!mbar_wait(smem_u32(&raw_full[r]), (it / RSTAGES) & 1, &abort_flag, poll_limit)) break;
      const unsigned char* rw = sbase + r * RAW_BYTES;
      unsigned char* sp = sbase + (st - base);
      int bad = 0;
      if (!TRANS) {
        // raw [128 rows][32 k]; pass p: rows 32p .. 32p+31, 8 threads per row
        float4 v[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const int f = p * NCONV + tid, m = f >> 3, k4 = f & 7;
          v[p] = *reinterpret_cast<const float4*>(rw + m * (TK * 4) + k4 * 16);
        }
        // the next TMA write (async proxy) must follow these generic reads
        fence_proxy_async();
        mbar_arrive(smem_u32(&raw_empty[r]));  // the raw stage is free for a later tile
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const int f = p * NCONV + tid, m = f >> 3, k4 = f & 7;
          const float sc = scs[p];
          float a[4] = {v[p].x * sc, v[p].y * sc, v[p].z * sc, v[p].w * sc};
          float sl[4][4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            bad |= !(fabsf(a[i]) < 128.f);
            cut4(a[i], sl[0][i], sl[1][i], sl[2][i], sl[3][i]);
          }
          const uint32_t off = sw64_off(m, k4 >> 1) + (uint32_t)((k4 & 1) * 8);
#pragma unroll
          for (int t = 0; t < NSL; ++t)
            *reinterpret_cast<uint2*>(sp + t * A_SLICE + off) =
                make_uint2(pack_bf16(sl[t][0], sl[t][1]), pack_bf16(sl[t][2], sl[t][3]));
        }
      } else {
        // raw [32 k][128 m]; thread (m, half) takes k = 16 half .. 16 half + 15
        const int m = tid & (TM - 1), h = tid >> 7;
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i)
          v[i] = *reinterpret_cast<const float*>(rw + ((h * 16 + i) * TM + m) * 4);
        fence_proxy_async();
        mbar_arrive(smem_u32(&raw_empty[r]));
        const float sc = scs[0];
#pragma unroll
        for (int q = 0; q < 2; ++q) {  // 16-byte chunk 2 h + q: k = 16 h + 8 q ..
          float sl[4][8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float a = v[q * 8 + i] * sc;
            bad |= !(fabsf(a) < 128.f);
            cut4(a, sl[0][i], sl[1][i], sl[2][i], sl[3][i]);
          }
          const uint32_t off = sw64_off(m, h * 2 + q);
#pragma unroll
          for (int t = 0; t < NSL; ++t)
            *reinterpret_cast<uint4*>(sp + t * A_SLICE + off) =
                make_uint4(pack_bf16(sl[t][0], sl[t][1]), pack_bf16(sl[t][2], sl[t][3]),
                           pack_bf16(sl[t][4], sl[t][5]), pack_bf16(sl[t][6], sl[t][7]));
        }
      }
      if (bad) abort_flag = 3;  // an entry outgrew its recorded row scale
      fence_proxy_async();
      mbar_arrive(smem_u32(&st_full[s]));
      ++it;
    }
  } else if (warp == W_XTMA) {
    // ---------------------------------------------------------- bulk copies of the X slices
    // the four pre-cut slices of a K tile are one contiguous 16 KB block of Xs,
    // already in the stage's swizzled order
    if (lane == 0) {
      const int64_t nkt_pad = 2 * ((n + KPAD - 1) / KPAD);  // K tiles of the padded Xs
      int it = 0;
      const uint64_t pol = l2_policy_evict_last();  // every row block re-reads X
      for (int kt = next_active(0); kt < nkt; kt = next_active(kt + 1)) {
        const int s = it % SSTAGES;
        if (!mbar_wait(smem_u32(&st_empty[s]), ((it / SSTAGES) & 1) ^ 1, &abort_flag, poll_limit))
          break;
        const uint32_t st = stage_addr0 + (uint32_t)s * STAGE_BYTES;
        mbar_arrive_tx(smem_u32(&x_full[s]), (uint32_t)(NSL * XB));
        const int64_t tile = (int64_t)ct * nkt_pad + kt;
        bulk_load_hint(st + NSL * A_SLICE + XZ * XB, Xs + tile * (NSL * TN * TK),
                       (uint32_t)(NSL * XB), smem_u32(&x_full[s]), pol);
        // the tile SSTAGES active tiles ahead, into L2 while this stage turns over
        int kp = kt;
        for (int i = 0; i < SSTAGES && kp < nkt; ++i) kp = next_active(kp + 1);
        if (kp < nkt)
          bulk_prefetch_l2(Xs + ((int64_t)ct * nkt_pad + kp) * (NSL * TN * TK),
                           (uint32_t)(NSL * XB));
        ++it;
      }
      for (int j = (it > SSTAGES ? it - SSTAGES : 0); j < it; ++j)
        mbar_wait_drain(smem_u32(&x_full[j % SSTAGES]), (j / SSTAGES) & 1);
    }
  } else if (warp == W_MMA) {
    // ---------------------------------------------------------- MMA issue
    if (lane == 0) {
      int it = 0, wc = 0, cur = -1;
      uint32_t started = 0, dbase = 0;
      bool ok = true;
      const uint32_t id = idesc_bf16_f32_n(NSL * TN);  // M = 128, N = 256
      for (int kt = next_active(0); kt < nkt && ok; kt = next_active(kt + 1)) {
        const int w = kt / WIN_TILES;
        if (w != cur) {
          if (cur >= 0) {
            mma_commit(smem_u32(&acc_full[wc & 1]));
            ++wc;
          }
          cur = w;
          ok = mbar_wait(smem_u32(&acc_empty[wc & 1]), ((wc >> 1) & 1) ^ 1, &abort_flag, poll_limit);
          if (!ok) break;
          dbase = tmem + (uint32_t)((wc & 1) * 4 * TN);
          started = 0;
        }
        const int s = it % SSTAGES;
        ok = mbar_wait(smem_u32(&st_full[s]), (it / SSTAGES) & 1, &abort_flag, poll_limit) &&
             mbar_wait(smem_u32(&x_full[s]), (it / SSTAGES) & 1, &abort_flag, poll_limit);
        if (!ok) break;
        tc_fence_after();
        const uint32_t st = stage_addr0 + (uint32_t)s * STAGE_BYTES;
        // descriptors of the stage's operands: the address field holds addr / 16
        // (the stage lies below 256 KB, so offsets add without carry)
        const uint64_t d0 = sw64_desc(st);
#pragma unroll
        for (int sa = 0; sa < NSL; ++sa) {
          // A slice sa + 1 times [0 .. x1 .. x(4 - sa)]: the 256 rows from block 3 - sa
          const uint64_t ad = d0 + (uint64_t)((sa * A_SLICE) >> 4);
          const uint64_t bd = d0 + (uint64_t)((NSL * A_SLICE + (XZ - sa) * XB) >> 4);
#pragma unroll
          for (int kk = 0; kk < TK / 16; ++kk) {  // K step kk is 32 bytes on
            mma_bf16(dbase, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), id, started);
            started = 1;
          }
        }
        mma_commit(smem_u32(&st_empty[s]));
        ++it;
      }
      if (ok && cur >= 0) mma_commit(smem_u32(&acc_full[wc & 1]));
      // every MMA issued by this thread completes before TMEM is released: this
      // wait ignores the other roles' abort and takes the full limit; only if
      // even that runs out is TMEM left allocated (the error flag reports it)
      mma_commit(smem_u32(&bar_final));
      if (!mbar_wait_drain(smem_u32(&bar_final), 0)) abort_flag = 2;
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
    int wc = 0;
    for (int w = 0; w < nwin; ++w) {
      int any = 0;
      for (int kt = w * WIN_TILES; kt < nkt && kt < (w + 1) * WIN_TILES; ++kt) any |= active(kt);
      if (!any) continue;
      const int b = wc & 1;
      const int exl = ex[((int64_t)w * nct + ct) * TN + half * 32 + lane];  // column lane
      const int ea = (m0 + r < n) ? e_rows[(m0 + r) * nwin + w] : 0;      // row, window
      if (!mbar_wait(smem_u32(&acc_full[b]), (wc >> 1) & 1, &abort_flag, poll_limit)) break;
      tc_fence_after();
      const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * 4 * TN + half * 32);
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        float sc[16], v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int e = ea + __shfl_sync(0xffffffffu, exl, g * 16 + j) - 14;
          sc[j] = (e >= -126 && e <= 127) ? pow2f(e) : ldexpf(1.f, e);
        }
        // orders 2..5: exact integer sums times exact powers of two, each added
        // into (hi, lo) through TwoSum, so that lo only gathers rounding residues
        // (the lower orders are not small: their digits run up to 128 against a
        // leading digit that may be much smaller)
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          const float cd = d == 0 ? 1.f : (d == 1 ? 0.00390625f : (d == 2 ? 1.52587890625e-05f
                                                                         : 5.9604644775390625e-08f));
          tmem_ld16(tl + (uint32_t)(d * TN + g * 16), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int jj = g * 16 + j;
            const float t = v[j] * (sc[j] * cd);
            const float sum = hi[jj] + t;
            const float bp = sum - hi[jj];
            lo[jj] += (hi[jj] - (sum - bp)) + (t - bp);
            hi[jj] = sum;
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&acc_empty[b]));
      ++wc;
    }
    const int64_t grow = m0 + r;
    const bool bad = abort_flag != 0;
    if (grow < n) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int64_t col = colbase + j;
        if (col < ncols) {
          const double v = bad ? __longlong_as_double(0x7ff8000000000000ll)
                               : (double)hi[j] + (double)lo[j];
          // split over K: Y was zeroed and every block adds its share
          if (gridDim.z > 1) atomicAdd(&Y[grow + col * ldy], v);
          else Y[grow + col * ldy] = v;
        }
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
// then one int exponent per (window, column) (sized per K tile, which is more)
int64_t gemm_esg_work_bytes(int64_t n, int64_t ncols) {
  const int64_t kpad = ((n + KPAD - 1) / KPAD) * KPAD;
  const int64_t nct = (ncols + TN - 1) / TN;
  const int64_t xs = nct * NSL * TN * kpad * 2;
  return ((xs + 255) / 256) * 256 + (kpad / TK) * nct * TN * 4;
}

int64_t gemm_esg_exp_count(int64_t n) { return n * ((n + WIN_ROWS - 1) / WIN_ROWS); }

void launch_esg_scales(const float* A, int64_t lda, int64_t n, int* aexp, cudaStream_t st) {
  count_launches(2);
  const int nw = (int)((n + WIN_ROWS - 1) / WIN_ROWS);
  k_row_exp<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(A, lda, n, nw, aexp);
  k_col_exp<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A, lda, n, nw, aexp + gemm_esg_exp_count(n));
}

int launch_gemm_esg(const float* A, int64_t lda, int trans, int64_t n, int64_t ncols,
                    const double* X, int64_t ldx, double* Y, int64_t ldy, void* work,
                    const int* aexp, uint8_t* flags, int* err, cudaStream_t st) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc::encode_fn();
  if (!enc || !gemm_tc_supported(A, lda, n)) return 1;
  const int64_t kpad = ((n + KPAD - 1) / KPAD) * KPAD;
  const int nct = (int)((ncols + TN - 1) / TN);
  const int nkt = (int)(kpad / TK);
  if (nkt > MAX_KT) return 1;
  __nv_bfloat16* Xs = (__nv_bfloat16*)work;
  const int64_t xs_bytes = (int64_t)nct * NSL * TN * kpad * 2;
  int* ex = (int*)((unsigned char*)work + ((xs_bytes + 255) / 256) * 256);
  CUtensorMap tmA;
  const cuuint64_t adim[2] = {(cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t astr[1] = {(cuuint64_t)lda * 4};
  const cuuint32_t abox[2] = {trans ? (cuuint32_t)TM : (cuuint32_t)TK,
                              trans ? (cuuint32_t)TK : (cuuint32_t)TM};
  const cuuint32_t one[2] = {1, 1};
  if (enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)A, adim, astr, abox, one,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 2;
  count_launches(2);
  const int nwin = (nkt + WIN_TILES - 1) / WIN_TILES;
  k_split_x64<<<dim3(nwin, nct), 256, 0, st>>>(X, ldx, n, ncols, kpad, nct, Xs, ex, flags);
  const int* e_rows = trans ? aexp + gemm_esg_exp_count(n) : aexp;
  const size_t smem = gemm_esg_smem_bytes();
  static std::atomic<uint32_t> done[2] = {{0}, {0}};
  // Split over K when the row blocks alone leave the last wave of blocks
  // (one per SM) markedly short: two blocks per row block share its windows,
  // each keeping >= 16 windows of the (typically half active) K range.  At most
  // two: two FP64 partials added into a zeroed Y give the same sum in either
  // order, so the results stay reproducible.
  const int nrb = (int)((n + TM - 1) / TM);
  int nsm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    nsm = 1;
  auto eff = [&](int k) {
    const int64_t c = (int64_t)nct * nrb * k;
    return (double)c / ((double)nsm * (double)((c + nsm - 1) / nsm));
  };
  int ks = 1;
  const int ks_max = std::max(1, std::min(2, nwin / 16));
  for (int k = 2; k <= ks_max; ++k)
    if (eff(k) > eff(ks) + 0.05) ks = k;
  if (ks > 1 &&
      cudaMemset2DAsync(Y, (size_t)ldy * sizeof(double), 0, (size_t)n * sizeof(double),
                        (size_t)ncols, st) != cudaSuccess)
    return 2;
  dim3 grid((unsigned)nct, (unsigned)nrb, (unsigned)ks);
  if (trans) {
    raise_smem_limit((const void*)k_gemm_esg<1, 0>, done[1]);
    k_gemm_esg<1, 0><<<grid, NTHREADS, smem, st>>>(tmA, Xs, n, ncols, flags, ex, e_rows, Y, ldy,
                                                   err, wait_limit(), nullptr, nullptr);
  } else {
    raise_smem_limit((const void*)k_gemm_esg<0, 0>, done[0]);
    k_gemm_esg<0, 0><<<grid, NTHREADS, smem, st>>>(tmA, Xs, n, ncols, flags, ex, e_rows, Y, ldy,
                                                   err, wait_limit(), nullptr, nullptr);
  }
  return 0;
}

}  // namespace hm

namespace hm {
namespace {

// The tables hold float pairs: S[0 .. n) high parts then S[n .. 2n) low parts,
// P[0 .. 2n - 1) high parts then P[2n - 1 .. 4n - 2) low parts.
// Exponents of the matrix-free log kernel per row and window of 256 columns: e
// with max |A(i, j)| < 2^e over the window (clamped to >= -120), the entries
// formed exactly as the generating cutters form them.  One warp per row.  The
// operator is symmetric: these are also the column exponents.
__global__ __launch_bounds__(256) void k_row_exp_logtab(const float* __restrict__ S,
                                                        const float* __restrict__ P, int64_t n,
                                                        int nw, int* __restrict__ e_row) {
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  for (int w = 0; w < nw; ++w) {
    float mx = 0.f;
    for (int64_t j = (int64_t)w * WIN_ROWS + lane; j < n && j < (int64_t)(w + 1) * WIN_ROWS;
         j += 32) {
      const int64_t d = row > j ? row - j : j - row;
      const float v = (d == 0) ? 1.f : (S[d] + P[row + j]) + (S[n + d] + P[2 * n - 1 + row + j]);
      mx = fmaxf(mx, fabsf(v));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) e_row[row * nw + w] = max(exp_above(mx), -120);
  }
}

// out[(i - r0) * ld + (j - c0)] = A(i, j) of the matrix-free log kernel.
__global__ void k_logtab_block(const float* __restrict__ S, const float* __restrict__ P,
                               int64_t n, int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                               float* __restrict__ out, int64_t ld) {
  for (int64_t i = r0 + blockIdx.y; i < r1; i += gridDim.y)
    for (int64_t j = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < c1;
         j += (int64_t)gridDim.x * blockDim.x) {
      const int64_t d = i > j ? i - j : j - i;
      out[(i - r0) * ld + (j - c0)] =
          (d == 0) ? 1.f : (S[d] + P[i + j]) + (S[n + d] + P[2 * n - 1 + i + j]);
    }
}

}  // namespace

void launch_logtab_rowexp(const float* S, const float* P, int64_t n, int* e_row, cudaStream_t st) {
  count_launches(1);
  k_row_exp_logtab<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(
      S, P, n, (int)((n + WIN_ROWS - 1) / WIN_ROWS), e_row);
}

void launch_logtab_block(const float* S, const float* P, int64_t n, int64_t r0, int64_t r1,
                         int64_t c0, int64_t c1, float* out, int64_t ld, cudaStream_t st) {
  count_launches(1);
  const int64_t w = c1 - c0, h = r1 - r0;
  dim3 grid((unsigned)std::min<int64_t>((w + 255) / 256, 1024),
            (unsigned)std::min<int64_t>(h, 65535));
  k_logtab_block<<<grid, 256, 0, st>>>(S, P, n, r0, r1, c0, c1, out, ld);
}

// Y = A X for the matrix-free log kernel (symmetric, so either product), FP64
// X and Y, with the exact-accumulation split of launch_gemm_esg; the entries of
// A are formed in the cutter warps from the tables S and P and never stored.
int launch_gemm_esg_gen(const float* S, const float* P, const int* rowexp, int64_t n,
                        int64_t ncols, const double* X, int64_t ldx, double* Y, int64_t ldy,
                        void* work, uint8_t* flags, int* err, cudaStream_t st) {
  const int64_t kpad = ((n + KPAD - 1) / KPAD) * KPAD;
  const int nct = (int)((ncols + TN - 1) / TN);
  const int nkt = (int)(kpad / TK);
  if (nkt > MAX_KT) return 1;
  __nv_bfloat16* Xs = (__nv_bfloat16*)work;
  const int64_t xs_bytes = (int64_t)nct * NSL * TN * kpad * 2;
  int* ex = (int*)((unsigned char*)work + ((xs_bytes + 255) / 256) * 256);
  // the kernel takes no TMA map of A in this form: a zeroed map fills the slot
  CUtensorMap tm0;
  memset(&tm0, 0, sizeof(tm0));
  count_launches(2);
  const int nwin = (nkt + WIN_TILES - 1) / WIN_TILES;
  k_split_x64<<<dim3(nwin, nct), 256, 0, st>>>(X, ldx, n, ncols, kpad, nct, Xs, ex, flags);
  const size_t smem = gemm_esg_smem_bytes();
  static std::atomic<uint32_t> done{0};
  // the same K split as the dense engine: two blocks share a row block's windows
  // when the grid's last wave is short
  const int nrb = (int)((n + TM - 1) / TM);
  int nsm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    nsm = 1;
  auto eff = [&](int k) {
    const int64_t c = (int64_t)nct * nrb * k;
    return (double)c / ((double)nsm * (double)((c + nsm - 1) / nsm));
  };
  int ks = 1;
  const int ks_max = std::max(1, std::min(2, nwin / 16));
  for (int k = 2; k <= ks_max; ++k)
    if (eff(k) > eff(ks) + 0.05) ks = k;
  if (ks > 1 &&
      cudaMemset2DAsync(Y, (size_t)ldy * sizeof(double), 0, (size_t)n * sizeof(double),
                        (size_t)ncols, st) != cudaSuccess)
    return 2;
  dim3 grid((unsigned)nct, (unsigned)nrb, (unsigned)ks);
  raise_smem_limit((const void*)k_gemm_esg<0, 1>, done);
  k_gemm_esg<0, 1><<<grid, NTHREADS, smem, st>>>(tm0, Xs, n, ncols, flags, ex, rowexp, Y, ldy,
                                                 err, wait_limit(), S, P);
  return 0;
}

}  // namespace hm
