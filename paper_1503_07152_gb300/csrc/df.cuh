// Double-float ("DF") arithmetic on the FP32 pipe: a value is the unevaluated
// sum hi + lo of two floats (about 48 significant bits).  GB300 runs FP64 at a
// small fraction of its FP32 rate, so the per-node factorizations of the HM_A32
// path (FP32 operator, FP64-accurate samples and bases) do their bulk work in
// this form.  The building blocks are the error-free transformations TwoSum
// (Knuth), FastTwoSum (Dekker) and TwoProduct by FMA; the compound operations
// follow the double-double algorithms of Dekker (1971) and Bailey's DD library
// carried over to float pairs.  nvcc does not reassociate floating-point adds
// without fast-math, which these transformations rely on.
#pragma once

namespace hm {
namespace df {

__device__ __forceinline__ void split(double x, float& h, float& l) {
  h = (float)x;
  l = (float)(x - (double)h);
}
__device__ __forceinline__ double join(float h, float l) { return (double)h + (double)l; }

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly when |a| >= |b| (Dekker's FastTwoSum)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// (h, l) += (bh, bl), renormalized
__device__ __forceinline__ void add_to(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e += l + bl;
  fast_two_sum(s, e, h, l);
}

// (sh, sl) += x * y for DF x, y: the leading product exactly by TwoProduct, the
// cross terms in FP32, the sum through TwoSum (the sum is left unnormalized:
// sl gathers the residues; add_to or join renormalize it)
__device__ __forceinline__ void dot_acc(float xh, float xl, float yh, float yl, float& sh,
                                        float& sl) {
  const float p = xh * yh;
  const float e = fmaf(xh, yl, fmaf(xl, yh, fmaf(xh, yh, -p)));
  float s, err;
  two_sum(sh, p, s, err);
  sh = s;
  sl += err + e;
}

// (h, l) = x * y
__device__ __forceinline__ void mul(float xh, float xl, float yh, float yl, float& h, float& l) {
  const float p = xh * yh;
  const float e = fmaf(xh, yl, fmaf(xl, yh, fmaf(xh, yh, -p)));
  fast_two_sum(p, e, h, l);
}

// (mh, ml) -= f * v
__device__ __forceinline__ void axpy_neg(float fh, float fl, float vh, float vl, float& mh,
                                         float& ml) {
  const float p = fh * vh;
  const float e = fmaf(fh, vl, fmaf(fl, vh, fmaf(fh, vh, -p)));
  float s, err;
  two_sum(mh, -p, s, err);
  err += ml - e;
  fast_two_sum(s, err, mh, ml);
}

// (h, l) = x - y
__device__ __forceinline__ void sub(float xh, float xl, float yh, float yl, float& h, float& l) {
  float s, e;
  two_sum(xh, -yh, s, e);
  e += xl - yl;
  fast_two_sum(s, e, h, l);
}

// (h, l) = sqrt(x) for x >= 0: the FP32 root s, then one Newton correction
// s + (x - s^2) / (2 s) with s^2 formed exactly (TwoProduct); about 2^-46
// relative (Karp and Markstein's form of the correction).
__device__ __forceinline__ void sqrt_df(float xh, float xl, float& h, float& l) {
  if (!(xh > 0.f)) { h = 0.f; l = 0.f; return; }
  const float s = sqrtf(xh);
  const float p = s * s;
  const float e = fmaf(s, s, -p);
  const float r = ((xh - p) - e) + xl;
  fast_two_sum(s, r * (0.5f / s), h, l);
}

// (h, l) = x / y (y != 0): the FP32 quotient q, then one correction with the
// exact remainder x - q y (TwoProduct); about 2^-46 relative.
__device__ __forceinline__ void div_df(float xh, float xl, float yh, float yl, float& h,
                                       float& l) {
  const float q = xh / yh;
  const float p = q * yh;
  const float e = fmaf(q, yh, -p);
  const float r = (((xh - p) - e) + xl) - q * yl;
  fast_two_sum(q, r / yh, h, l);
}

// DF sum over a warp (xor butterfly): every lane ends with the total
__device__ __forceinline__ void warp_sum(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    add_to(h, l, oh, ol);
  }
}
// the same over aligned groups of 8 lanes
__device__ __forceinline__ void group8_sum(float& h, float& l) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    add_to(h, l, oh, ol);
  }
}

}  // namespace df
}  // namespace hm
