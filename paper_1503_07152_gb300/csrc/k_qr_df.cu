// FP64-accurate SVD of the panels' R factors in double-float arithmetic
// (HM_A32): the phases of k_jacobi_mp (k_qr.cu) with every bulk FP64 operation
// carried by float pairs on the FP32 pipe, which GB300 runs at many times its
// FP64 rate.  Inputs and outputs stay FP64.
#include <atomic>

#include "df.cuh"
#include "hm_internal.h"

namespace hm {
namespace {

// (xh, xl) <- c x - s y and (yh, yl) <- s x + c y for DF c, s, x, y: the leading
// products exactly by TwoProduct, the cross terms in FP32, one TwoSum and a
// renormalization per output.
__device__ __forceinline__ void rot_df(float ch, float cl, float sh, float sl, float& xh, float& xl,
                                       float& yh, float& yl) {
  const float x0 = xh, x1 = xl, y0 = yh, y1 = yl;
  {
    const float p1 = ch * x0, p2 = sh * y0;
    const float e1 = fmaf(ch, x0, -p1), e2 = fmaf(sh, y0, -p2);
    float r, e3;
    df::two_sum(p1, -p2, r, e3);
    float lo = (e1 - e2) + e3;
    lo = fmaf(ch, x1, fmaf(cl, x0, lo));
    lo = fmaf(-sh, y1, fmaf(-sl, y0, lo));
    df::fast_two_sum(r, lo, xh, xl);
  }
  {
    const float p1 = sh * x0, p2 = ch * y0;
    const float e1 = fmaf(sh, x0, -p1), e2 = fmaf(ch, y0, -p2);
    float r, e3;
    df::two_sum(p1, p2, r, e3);
    float lo = (e1 + e2) + e3;
    lo = fmaf(sh, x1, fmaf(sl, x0, lo));
    lo = fmaf(ch, y1, fmaf(cl, y0, lo));
    df::fast_two_sum(r, lo, yh, yl);
  }
}

// Rotation of one FP32 Jacobi pair (phase B below): ga = a_p . a_q, al and be
// the squared norms.  Flags a correlation above big2 (another sweep is due) and
// returns false when the pair is already orthogonal to tol; otherwise (tc, ts)
// = (cos, sin) of the angle that zeroes ga (the smaller root of the standard
// two-sided formula).
__device__ __forceinline__ bool jacobi_angle32(float ga, float al, float be, float tol,
                                               float big2, int gl, int& large, float& tc,
                                               float& ts) {
  if (gl == 0 && al > 0.f && be > 0.f && (ga / al) * (ga / be) > big2) large = 1;
  if (!(ga != 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be))) return false;
  const float zeta = (be - al) / (2.f * ga);
  const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  tc = 1.f / sqrtf(1.f + t * t);
  ts = tc * t;
  return true;
}
// the pair's squared norms after the rotation (c^2 al - 2cs ga + s^2 be and
// s^2 al + 2cs ga + c^2 be, clamped at 0)
__device__ __forceinline__ void jacobi_norms32(float tc, float ts, float ga, float& np,
                                               float& nq) {
  const float al = np, be = nq;
  const float cs2 = 2.f * tc * ts, c2 = tc * tc, s2 = ts * ts;
  np = fmaxf(fmaf(c2, al, fmaf(-cs2, ga, s2 * be)), 0.f);
  nq = fmaxf(fmaf(s2, al, fmaf(cs2, ga, c2 * be)), 0.f);
}

// SVD of R (c x c, c <= 128) to about 2^-46 relative accuracy for HM_A32, the
// phases of k_jacobi_mp with every bulk FP64 operation in double-float:
//   A. column-pivoted Householder QR R P = Q2 R2 (Businger-Golub; DF entries,
//      column norms and reflector scalars in FP64); X = R2^T (graded columns)
//      parked in the node's W slot;
//   B. one-sided Jacobi on float(X), rotations accumulated into V32 (FP32);
//   C. Q = classical Gram-Schmidt of V32 in DF;
//   D. X1 = X Q in DF: the left singular vectors of X, columns orthogonal to
//      FP32 precision;
//   E. one-sided Jacobi sweeps on X1 in DF until every pair's correlation is
//      below the DF rounding level (angles from FP32 ratios of DF quantities:
//      small-angle series for |t| < 2^-11, FP64 formulas otherwise; the
//      rotations themselves in DF, orthogonal to DF rounding);
//   F. sigma_j = |X1_j|, W = P U_x from the normalized columns, sorted
//      descending, the sign convention of k_jacobi_mp.
// R is scaled by a power of two (exact) so that its largest entry lies in
// [1, 2): squared column norms then stay inside the float range.
__global__ __launch_bounds__(512, 1) void k_jacobi_df(const int32_t* __restrict__ node_slot,
                                                      const double* __restrict__ R, int c,
                                                      double* __restrict__ W,
                                                      double* __restrict__ sigma,
                                                      const NodeJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const double* Rs;
  double *Wn, *sig;
  if (jobs) {  // a level-wide launch over several operators' nodes
    const NodeJob& jb = jobs[blockIdx.x];
    c = jb.c;
    Rs = jb.R;
    Wn = jb.W;
    sig = jb.sigma;
  } else {
    Rs = R + (int64_t)node_slot[blockIdx.x] * c * c;
    Wn = W + (int64_t)blockIdx.x * c * c;
    sig = sigma + (int64_t)blockIdx.x * c;
  }
  const int cc = c * c;
  float* reg0 = reinterpret_cast<float*>(smem_raw);
  float* reg1 = reg0 + cc;
  float* reg2 = reg1 + cc;
  float* Mh = reg0;   // A: R, then R2 (column-major)
  float* Ml = reg1;
  float* V32 = reg0;  // B, C
  float* X32 = reg1;  // B
  float* Qh = reg1;   // C - F
  float* Ql = reg2;
  __shared__ int rotated, large;
  __shared__ double sv[128], hb[128];
  __shared__ float cnh[128], cnl[128], hbh[128], hbl[128];
  __shared__ float psh[4][128], psl[4][128];
  __shared__ int perm[128], order[128];
  __shared__ signed char sgn[128];
  __shared__ double red_v[16];
  __shared__ int red_i[16];
  __shared__ float pnh[128], pnl[128], ph0[128];  // A: pivoting norms
  __shared__ float sh_ah, sh_al, sh_sh, sh_sl;
  __shared__ int sh_exp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int nthr = blockDim.x;
  const int pg = tid >> 3, gl = tid & 7;
  // ------------------------------------------------------------- scale
  {
    double mx = 0.0;
    for (int idx = tid; idx < cc; idx += nthr) mx = fmax(mx, fabs(Rs[idx]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red_v[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = 0.0;
      for (int w = 0; w < nwarps; ++w) m2 = fmax(m2, red_v[w]);
      int e = 0;
      if (m2 > 0.0 && isfinite(m2)) frexp(m2, &e);  // m2 in [2^(e-1), 2^e)
      sh_exp = e - 1;
    }
    __syncthreads();
  }
  const int ex = sh_exp;
  // ---------------------------------------------------------------- A
  for (int idx = tid; idx < cc; idx += nthr) {
    const int rr = idx / c, col = idx % c;
    df::split(ldexp(Rs[idx], -ex), Mh[col * c + rr], Ml[col * c + rr]);
  }
  for (int j = tid; j < c; j += nthr) perm[j] = j;
  __syncthreads();
  // Squared column norms for the pivoting, kept as double-float pairs (pnh, pnl)
  // and downdated per step; ph0 holds the value at the last exact recompute.
  // Every scalar of this phase is double-float: a dependent chain of FP64
  // instructions (a square root, a division) is very long on GB300's FP64 pipe.
  for (int k = warp; k < c; k += nwarps) {
    float sh = 0.f, sl = 0.f;
    for (int i = lane; i < c; i += 32) df::dot_acc(Mh[k * c + i], Ml[k * c + i], Mh[k * c + i], Ml[k * c + i], sh, sl);
    df::warp_sum(sh, sl);
    if (lane == 0) { df::fast_two_sum(sh, sl, pnh[k], pnl[k]); ph0[k] = pnh[k]; }
  }
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    // recompute the norms that downdating has left with few correct digits
    for (int k = j + warp; k < c; k += nwarps) {
      if (!(pnh[k] > 5.9604644775390625e-08f * ph0[k])) {
        float sh = 0.f, sl = 0.f;
        for (int i = j + lane; i < c; i += 32)
          df::dot_acc(Mh[k * c + i], Ml[k * c + i], Mh[k * c + i], Ml[k * c + i], sh, sl);
        df::warp_sum(sh, sl);
        if (lane == 0) { df::fast_two_sum(sh, sl, pnh[k], pnl[k]); ph0[k] = pnh[k]; }
      }
    }
    __syncthreads();
    if (warp == 0) {  // the largest remaining norm, the first on ties
      float bh = -1.f, bl = 0.f;
      int bi = c;
      for (int k = j + lane; k < c; k += 32)
        if (pnh[k] > bh || (pnh[k] == bh && pnl[k] > bl)) { bh = pnh[k]; bl = pnl[k]; bi = k; }
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, bh, o);
        const float ol = __shfl_xor_sync(0xffffffffu, bl, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oh > bh || (oh == bh && (ol > bl || (ol == bl && oi < bi)))) { bh = oh; bl = ol; bi = oi; }
      }
      if (lane == 0) red_i[0] = bi;
    }
    __syncthreads();
    const int p = red_i[0];
    if (p != j && p < c) {
      for (int i = tid; i < c; i += nthr) {
        float t = Mh[j * c + i]; Mh[j * c + i] = Mh[p * c + i]; Mh[p * c + i] = t;
        t = Ml[j * c + i]; Ml[j * c + i] = Ml[p * c + i]; Ml[p * c + i] = t;
      }
      if (tid == 0) {
        const int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
        float u = pnh[j]; pnh[j] = pnh[p]; pnh[p] = u;
        u = pnl[j]; pnl[j] = pnl[p]; pnl[p] = u;
        u = ph0[j]; ph0[j] = ph0[p]; ph0[p] = u;
      }
    }
    __syncthreads();
    float* mjh = Mh + j * c;
    float* mjl = Ml + j * c;
    if (warp == 0) {  // the reflector needs the pivot column's exact norm
      float sh = 0.f, sl = 0.f;
      for (int i = j + lane; i < c; i += 32) df::dot_acc(mjh[i], mjl[i], mjh[i], mjl[i], sh, sl);
      df::warp_sum(sh, sl);
      if (lane == 0) {
        // x0 and the reflector scale sqrt(2 / v^T v), v^T v = 2 nrm (nrm + |x0|)
        const float xh = mjh[j], xl = mjl[j];
        float nh, nl;
        df::sqrt_df(sh, sl, nh, nl);
        const float ah = (xh > 0.f) ? -nh : nh, al = (xh > 0.f) ? -nl : nl;
        float vh, vl, wh = nh, wl = nl, qh, ql, sch = 0.f, scl = 0.f;
        df::sub(xh, xl, ah, al, vh, vl);                        // v0 = x0 - alpha
        df::add_to(wh, wl, fabsf(xh), xh < 0.f ? -xl : xl);      // nrm + |x0|
        df::mul(nh, nl, wh, wl, qh, ql);                         // v^T v / 2
        if (qh > 0.f) {
          float ih, il;
          df::div_df(1.f, 0.f, qh, ql, ih, il);
          df::sqrt_df(ih, il, sch, scl);
        }
        sh_ah = ah;
        sh_al = al;
        sh_sh = sch;
        sh_sl = scl;
        df::mul(vh, vl, sch, scl, mjh[j], mjl[j]);
      }
    }
    __syncthreads();
    const float sch = sh_sh, scl = sh_sl;
    for (int i = j + 1 + tid; i < c; i += nthr) df::mul(sch, scl, mjh[i], mjl[i], mjh[i], mjl[i]);
    __syncthreads();
    if (sch != 0.f) {
      for (int k0 = j + 1; k0 < c; k0 += 64) {  // one 8-lane group per trailing column
        const int k = k0 + pg;
        const bool on = k < c;
        float* mkh = Mh + (on ? k : j) * c;
        float* mkl = Ml + (on ? k : j) * c;
        float dh = 0.f, dl = 0.f;
        if (on) {
#pragma unroll
          for (int ii = 0; ii < 16; ++ii) {
            const int i = j + gl + 8 * ii;
            if (i < c) df::dot_acc(mjh[i], mjl[i], mkh[i], mkl[i], dh, dl);
          }
        }
        df::group8_sum(dh, dl);
        if (on) {
          float fh, fl;
          df::fast_two_sum(dh, dl, fh, fl);
#pragma unroll
          for (int ii = 0; ii < 16; ++ii) {
            const int i = j + gl + 8 * ii;
            if (i < c) df::axpy_neg(fh, fl, mjh[i], mjl[i], mkh[i], mkl[i]);
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && sch != 0.f) { mjh[j] = sh_ah; mjl[j] = sh_al; }
    for (int k = j + 1 + tid; k < c; k += nthr) {  // downdate: |col k|^2 -= R(j, k)^2
      float rh, rl;
      df::mul(Mh[k * c + j], Ml[k * c + j], Mh[k * c + j], Ml[k * c + j], rh, rl);
      df::sub(pnh[k], pnl[k], rh, rl, pnh[k], pnl[k]);
    }
    __syncthreads();
  }
  // X = R2^T, column-major, parked in the W slot as float pairs (hi parts, then
  // lo parts: the c x c doubles of the slot hold both), so that phase D reads it
  // without conversions
  float* Xph = reinterpret_cast<float*>(Wn);
  float* Xpl = Xph + cc;
  for (int idx = tid; idx < cc; idx += nthr) {
    const int col = idx / c, row = idx % c;  // X(row, col) = R2(col, row), zero above
    const bool low = row >= col;
    Xph[idx] = low ? Mh[row * c + col] : 0.f;
    Xpl[idx] = low ? Ml[row * c + col] : 0.f;
  }
  __syncthreads();
  // ---------------------------------------------------------------- B
  for (int idx = tid; idx < cc; idx += nthr) {
    X32[idx] = Xph[idx];
    V32[idx] = (idx / c == idx % c) ? 1.f : 0.f;
  }
  __syncthreads();
  const int cp = (c + 1) & ~1;
  float* cn32 = cnh;  // FP32 squared column norms of X32 (cnh is free until E)
  for (int j = warp; j < c; j += nwarps) {
    float s2 = 0.f;
    for (int i = lane; i < c; i += 32) s2 = fmaf(X32[j * c + i], X32[j * c + i], s2);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) cn32[j] = s2;
  }
  __syncthreads();
  {
    // (element loops over a fixed 16 strided elements per lane, c <= 128, so
    // that they unroll; the arithmetic and its order are those of the plain loops)
    const float tol = (float)(5.960464477539063e-08 * sqrt((double)c));
    const float big2 = tol;
    const bool vec = (c & 3) == 0;
    for (int sweep = 0; sweep < 40; ++sweep) {
      if (tid == 0) { rotated = 0; large = 0; }
      __syncthreads();
      for (int step = 0; step < cp - 1; ++step) {
        int p = c, q = c;
        if (pg < cp / 2) {
          const int a = pg, b = cp - 1 - pg;
          // round-robin pairing: a - 1 + step < 2 (cp - 1) and b - 1 + step < 2 (cp - 1)
          int va = a - 1 + step, vb = b - 1 + step;
          if (va >= cp - 1) va -= cp - 1;
          if (vb >= cp - 1) vb -= cp - 1;
          p = (a == 0) ? 0 : va + 1;
          q = vb + 1;
        }
        const bool valid = p < c && q < c;
        float* ap = X32 + (valid ? p : 0) * c;
        float* aq = X32 + (valid ? q : 0) * c;
        if (vec) {
          // c a multiple of 4: lane gl holds the 16-byte chunks gl, gl + 8, ..
          // of both columns in registers (one 128-byte row of shared memory per
          // group and load: no bank conflicts) for the dot product and the
          // rotation
          const int c4 = c >> 2;
          float4 xa[4], xb[4];
          float ga = 0.f;
          if (valid) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int ch = gl + 8 * k;
              if (ch < c4) {
                xa[k] = reinterpret_cast<const float4*>(ap)[ch];
                xb[k] = reinterpret_cast<const float4*>(aq)[ch];
                ga = fmaf(xa[k].x, xb[k].x, ga);
                ga = fmaf(xa[k].y, xb[k].y, ga);
                ga = fmaf(xa[k].z, xb[k].z, ga);
                ga = fmaf(xa[k].w, xb[k].w, ga);
              }
            }
          }
          ga += __shfl_xor_sync(0xffffffffu, ga, 4);
          ga += __shfl_xor_sync(0xffffffffu, ga, 2);
          ga += __shfl_xor_sync(0xffffffffu, ga, 1);
          float tc, ts;
          if (valid && jacobi_angle32(ga, cn32[p], cn32[q], tol, big2, gl, large, tc, ts)) {
            float4* vp = reinterpret_cast<float4*>(V32 + p * c);
            float4* vq = reinterpret_cast<float4*>(V32 + q * c);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int ch = gl + 8 * k;
              if (ch < c4) {
                const float4 x = xa[k], y = xb[k];
                reinterpret_cast<float4*>(ap)[ch] =
                    make_float4(tc * x.x - ts * y.x, tc * x.y - ts * y.y, tc * x.z - ts * y.z,
                                tc * x.w - ts * y.w);
                reinterpret_cast<float4*>(aq)[ch] =
                    make_float4(ts * x.x + tc * y.x, ts * x.y + tc * y.y, ts * x.z + tc * y.z,
                                ts * x.w + tc * y.w);
                const float4 u = vp[ch], w = vq[ch];
                vp[ch] = make_float4(tc * u.x - ts * w.x, tc * u.y - ts * w.y,
                                     tc * u.z - ts * w.z, tc * u.w - ts * w.w);
                vq[ch] = make_float4(ts * u.x + tc * w.x, ts * u.y + tc * w.y,
                                     ts * u.z + tc * w.z, ts * u.w + tc * w.w);
              }
            }
            __syncwarp(0xffu << (8 * (lane >> 3)));  // the group's reads of the norms first
            if (gl == 0) {
              jacobi_norms32(tc, ts, ga, cn32[p], cn32[q]);
              rotated = 1;
            }
          }
        } else {
          float ga = 0;
          if (valid) {
#pragma unroll
            for (int ii = 0; ii < 16; ++ii) {
              const int i = gl + 8 * ii;
              if (i < c) ga = fmaf(ap[i], aq[i], ga);
            }
          }
          ga += __shfl_xor_sync(0xffffffffu, ga, 4);
          ga += __shfl_xor_sync(0xffffffffu, ga, 2);
          ga += __shfl_xor_sync(0xffffffffu, ga, 1);
          float tc, ts;
          if (valid && jacobi_angle32(ga, cn32[p], cn32[q], tol, big2, gl, large, tc, ts)) {
            float* vp = V32 + p * c;
            float* vq = V32 + q * c;
#pragma unroll
            for (int ii = 0; ii < 16; ++ii) {
              const int i = gl + 8 * ii;
              if (i < c) {
                const float x = ap[i], y = aq[i];
                ap[i] = tc * x - ts * y;
                aq[i] = ts * x + tc * y;
              }
            }
#pragma unroll
            for (int ii = 0; ii < 16; ++ii) {
              const int i = gl + 8 * ii;
              if (i < c) {
                const float x = vp[i], y = vq[i];
                vp[i] = tc * x - ts * y;
                vq[i] = ts * x + tc * y;
              }
            }
            __syncwarp(0xffu << (8 * (lane >> 3)));  // the group's reads of the norms first
            if (gl == 0) {
              jacobi_norms32(tc, ts, ga, cn32[p], cn32[q]);
              rotated = 1;
            }
          }
        }
        __syncthreads();
      }
      const int any = rotated && large;
      __syncthreads();
      if (!any) break;
    }
  }
  // ---------------------------------------------------------------- C
  // (X32 is dead; Q overlays it and the third region)
  for (int j = 0; j < c; ++j) {
    float* qjh = Qh + j * c;
    float* qjl = Ql + j * c;
    for (int i = tid; i < c; i += nthr) { qjh[i] = V32[j * c + i]; qjl[i] = 0.f; }
    __syncthreads();
    for (int i0 = 0; i0 < j; i0 += 64) {  // one 8-lane group per earlier column
      const int i = i0 + pg;
      const bool on = i < j;
      const float* qih = Qh + (on ? i : 0) * c;
      const float* qil = Ql + (on ? i : 0) * c;
      float sh = 0.f, sl = 0.f;
      if (on) {
#pragma unroll
        for (int ee = 0; ee < 16; ++ee) {
          const int e = gl + 8 * ee;
          if (e < c) df::dot_acc(qih[e], qil[e], qjh[e], qjl[e], sh, sl);
        }
      }
      df::group8_sum(sh, sl);
      if (on && gl == 0) { hbh[i] = sh; hbl[i] = sl; }
    }
    __syncthreads();
    {  // q_j -= sum_i hb[i] Q_i in four partial sums over quarters of i
      const int e = tid & 127, part = tid >> 7;
      const int i0 = (j * part) >> 2, i1 = (j * (part + 1)) >> 2;
      float sh = 0.f, sl = 0.f;
      if (e < c)
        for (int i = i0; i < i1; ++i) df::dot_acc(hbh[i], hbl[i], Qh[i * c + e], Ql[i * c + e], sh, sl);
      df::add_to(sh, sl, 0.f, 0.f);
      psh[part][e] = sh;
      psl[part][e] = sl;
    }
    __syncthreads();
    for (int e = tid; e < c; e += nthr) {
      float sh = psh[0][e], sl = psl[0][e];
      df::add_to(sh, sl, psh[1][e], psl[1][e]);
      df::add_to(sh, sl, psh[2][e], psl[2][e]);
      df::add_to(sh, sl, psh[3][e], psl[3][e]);
      df::add_to(qjh[e], qjl[e], -sh, -sl);
    }
    __syncthreads();
    if (warp == 0) {
      float sh = 0.f, sl = 0.f;
      for (int e = lane; e < c; e += 32) df::dot_acc(qjh[e], qjl[e], qjh[e], qjl[e], sh, sl);
      df::warp_sum(sh, sl);
      if (lane == 0) {
        const double s = df::join(sh, sl);
        df::split((s > 0.0) ? 1.0 / sqrt(s) : 0.0, sh_sh, sh_sl);
      }
    }
    __syncthreads();
    const float ih = sh_sh, il = sh_sl;
    for (int e = tid; e < c; e += nthr) df::mul(ih, il, qjh[e], qjl[e], qjh[e], qjl[e]);
    __syncthreads();
  }
  // ---------------------------------------------------------------- D
  for (int j = warp; j < c; j += nwarps) {
    float ah[4] = {0.f, 0.f, 0.f, 0.f}, alo[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < c; ++k) {
      const float qh = Qh[j * c + k], ql = Ql[j * c + k];
      const float* xkh = Xph + k * c;
      const float* xkl = Xpl + k * c;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int row = lane + 32 * rr;
        if (row < c) df::dot_acc(xkh[row], xkl[row], qh, ql, ah[rr], alo[rr]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int row = lane + 32 * rr;
      if (row < c) df::fast_two_sum(ah[rr], alo[rr], Qh[j * c + row], Ql[j * c + row]);
    }
  }
  __syncthreads();
  // ---------------------------------------------------------------- E
  for (int j = warp; j < c; j += nwarps) {
    float sh = 0.f, sl = 0.f;
    for (int i = lane; i < c; i += 32) df::dot_acc(Qh[j * c + i], Ql[j * c + i], Qh[j * c + i], Ql[j * c + i], sh, sl);
    df::warp_sum(sh, sl);
    if (lane == 0) df::fast_two_sum(sh, sl, cnh[j], cnl[j]);
  }
  __syncthreads();
  {
    // a pair is rotated while its correlation exceeds the DF rounding level of
    // the length-c dot products that measure it
    const float tol = (float)(3.552713678800501e-15 * sqrt((double)c));  // 2^-48 sqrt(c)
    const float tol2 = tol * tol, big2 = tol;
    for (int sweep = 0; sweep < 12; ++sweep) {
      if (tid == 0) { rotated = 0; large = 0; }
      __syncthreads();
      for (int step = 0; step < cp - 1; ++step) {
        int p = c, q = c;
        if (pg < cp / 2) {
          const int a = pg, b = cp - 1 - pg;
          int va = a - 1 + step, vb = b - 1 + step;
          if (va >= cp - 1) va -= cp - 1;
          if (vb >= cp - 1) vb -= cp - 1;
          p = (a == 0) ? 0 : va + 1;
          q = vb + 1;
        }
        const bool valid = p < c && q < c;
        float* aph = Qh + (valid ? p : 0) * c;
        float* apl = Ql + (valid ? p : 0) * c;
        float* aqh = Qh + (valid ? q : 0) * c;
        float* aql = Ql + (valid ? q : 0) * c;
        float gh = 0.f, glo = 0.f;
        if (valid) {
#pragma unroll
          for (int ii = 0; ii < 16; ++ii) {
            const int i = gl + 8 * ii;
            if (i < c) df::dot_acc(aph[i], apl[i], aqh[i], aql[i], gh, glo);
          }
        }
        df::group8_sum(gh, glo);
        df::fast_two_sum(gh, glo, gh, glo);
        if (valid) {
          const float al = cnh[p], be = cnh[q];
          const bool live = al > 0.f && be > 0.f && gh != 0.f;
          const float r2 = live ? (gh / al) * (gh / be) : 0.f;  // correlation squared
          if (gl == 0 && r2 > big2) large = 1;
          if (r2 > tol2) {
            const float d = (be - al) + (cnl[q] - cnl[p]);
            float ch, cl, sh, sl;
            if (fabsf(gh) < 0.00048828125f * fabsf(d)) {  // |t| < 2^-11
              const float u = gh / d;                       // 1 / (2 zeta)
              const float t = fmaf(-u * u, u, u);           // tan(theta) = u - u^3 + ...
              const float t2 = t * t;
              ch = 1.f;
              cl = t2 * fmaf(t2, 0.375f, -0.5f);            // cos - 1 = -t^2/2 + 3t^4/8
              sh = t;
              sl = t * cl;                                  // sin = t cos
            } else {  // |zeta| <= 2^10 here: zeta^2 stays in float range
              float zh, zl, th, tl, uh, ul;
              df::sub(be, cnl[q], al, cnl[p], uh, ul);             // |a_q|^2 - |a_p|^2
              df::div_df(uh, ul, 2.f * gh, 2.f * glo, zh, zl);     // zeta
              df::mul(zh, zl, zh, zl, th, tl);
              df::add_to(th, tl, 1.f, 0.f);
              df::sqrt_df(th, tl, uh, ul);                         // sqrt(1 + zeta^2)
              df::add_to(uh, ul, fabsf(zh), zh < 0.f ? -zl : zl);
              df::div_df(zh >= 0.f ? 1.f : -1.f, 0.f, uh, ul, th, tl);  // t = tan(theta)
              df::mul(th, tl, th, tl, uh, ul);
              df::add_to(uh, ul, 1.f, 0.f);
              float rh, rl;
              df::sqrt_df(uh, ul, rh, rl);
              df::div_df(1.f, 0.f, rh, rl, ch, cl);               // cos = 1 / sqrt(1 + t^2)
              df::mul(ch, cl, th, tl, sh, sl);                     // sin = t cos
            }
#pragma unroll
            for (int ii = 0; ii < 16; ++ii) {
              const int i = gl + 8 * ii;
              if (i < c) rot_df(ch, cl, sh, sl, aph[i], apl[i], aqh[i], aql[i]);
            }
            if (gl == 0) {
              // norms after the rotation: c^2 al - 2cs ga + s^2 be, s^2 al + 2cs ga + c^2 be
              float c2h, c2l, s2h, s2l, csh, csl, th, tl;
              df::mul(ch, cl, ch, cl, c2h, c2l);
              df::mul(sh, sl, sh, sl, s2h, s2l);
              df::mul(ch, cl, sh, sl, csh, csl);
              csh *= 2.f;
              csl *= 2.f;
              const float alh = cnh[p], all = cnl[p], beh = cnh[q], bel = cnl[q];
              float ph = 0.f, pl = 0.f, qh = 0.f, ql = 0.f;
              df::mul(c2h, c2l, alh, all, ph, pl);
              df::mul(csh, csl, gh, glo, th, tl);
              df::add_to(ph, pl, -th, -tl);
              df::mul(s2h, s2l, beh, bel, th, tl);
              df::add_to(ph, pl, th, tl);
              df::mul(s2h, s2l, alh, all, qh, ql);
              df::mul(csh, csl, gh, glo, th, tl);
              df::add_to(qh, ql, th, tl);
              df::mul(c2h, c2l, beh, bel, th, tl);
              df::add_to(qh, ql, th, tl);
              cnh[p] = ph; cnl[p] = pl;
              cnh[q] = qh; cnl[q] = ql;
              rotated = 1;
            }
          }
        }
        __syncthreads();
      }
      const int any = rotated && large;
      __syncthreads();
      if (!any) break;
    }
  }
  // ---------------------------------------------------------------- F
  for (int j = warp; j < c; j += nwarps) {
    float sh = 0.f, sl = 0.f;
    for (int i = lane; i < c; i += 32) df::dot_acc(Qh[j * c + i], Ql[j * c + i], Qh[j * c + i], Ql[j * c + i], sh, sl);
    df::warp_sum(sh, sl);
    if (lane == 0) {
      const double s = df::join(sh, sl);
      sv[j] = isfinite(s) ? sqrt(s) : -1.0;
    }
  }
  __syncthreads();
  for (int j = tid; j < c; j += nthr) {
    int rk = 0;
    for (int i = 0; i < c; ++i) rk += (sv[i] > sv[j]) || (sv[i] == sv[j] && i < j);
    order[rk] = j;
  }
  __syncthreads();
  for (int j = warp; j < c; j += nwarps) {
    const float* xh = Qh + order[j] * c;
    const float* xl = Ql + order[j] * c;
    double best = -1.0, bv = 0.0;
    int bi = c;
    for (int i = lane; i < c; i += 32) {
      const double x = df::join(xh[i], xl[i]);
      const double a = fabs(x);
      const int row = perm[i];
      if (a > best || (a == best && row < bi)) { best = a; bi = row; bv = x; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; bv = ov; }
    }
    if (lane == 0) {
      sgn[j] = (bv < 0.0) ? -1 : 1;
      hb[j] = (sv[order[j]] > 0.0) ? 1.0 / sv[order[j]] : 0.0;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < cc; idx += nthr) {
    const int i = idx % c, col = idx / c;
    const int j = order[col];
    const double u = df::join(Qh[j * c + i], Ql[j * c + i]) * hb[col];
    Wn[perm[i] + col * c] = sgn[col] < 0 ? -u : u;
  }
  for (int j = tid; j < c; j += nthr)
    sig[j] = sv[order[j]] > 0.0 ? ldexp(sv[order[j]], ex) : 0.0;
}


constexpr int TQ_THREADS = 512;  // threads of the double-float TSQR kernels

// Householder QR of one row block of a panel (the first TSQR round, <= 128 rows,
// FP64 data) in double-float: the steps of k_tsqr with every operation (the
// norms, the reflector's scalars, the dot products and updates of the trailing
// columns) carried by float pairs on the FP32 pipe.  v^T v is formed as
// 2 nrm (nrm + |x0|), the cancellation-free form of |x|^2 - x0^2 + v0^2.
// Writes the c x c R (row-major, upper triangle) in FP64.
__global__ __launch_bounds__(TQ_THREADS) void k_tsqr_df(const TsqrTask* __restrict__ tasks,
                                                 const double* __restrict__ P, int64_t ldp,
                                                 int c, double* __restrict__ R, int ldm,
                                                 const NodeJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TsqrTask* tkp = tasks + blockIdx.x;
  if (jobs) {  // a level-wide launch over several operators' nodes
    const NodeJob& jb = jobs[blockIdx.x];
    tkp = jb.task;
    P = jb.P;
    ldp = jb.ldp;
    c = jb.c;
    R = jb.R;
  }
  const TsqrTask tk = *tkp;
  float* Mh = reinterpret_cast<float*>(smem_raw);  // column-major, ld = ldm, high parts
  float* Ml = Mh + (size_t)ldm * c;                 // low parts
  __shared__ float red_h[TQ_THREADS / 32], red_l[TQ_THREADS / 32];
  __shared__ float sh_ah, sh_al, sh_bh, sh_bl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int m = 0;
  for (int s = 0; s < tk.nsrc; ++s) {
    if (tk.kind[s] == 0) {
      const int rows = (int)(tk.r1[s] - tk.r0[s]);
      for (int idx = tid; idx < rows * c; idx += TQ_THREADS) {
        const int rr = idx % rows, col = idx / rows;
        df::split(P[tk.r0[s] + rr + (int64_t)col * ldp], Mh[col * ldm + m + rr],
                  Ml[col * ldm + m + rr]);
      }
      m += rows;
    } else {
      const double* Rs = R + (int64_t)tk.slot[s] * c * c;
      for (int idx = tid; idx < c * c; idx += TQ_THREADS) {
        const int rr = idx / c, col = idx % c;
        df::split(Rs[rr * c + col], Mh[col * ldm + m + rr], Ml[col * ldm + m + rr]);
      }
      m += c;
    }
  }
  __syncthreads();
  const int steps = m < c ? m : c;
  for (int j = 0; j < steps; ++j) {
    float* mjh = Mh + j * ldm;
    float* mjl = Ml + j * ldm;
    float sh = 0.f, sl = 0.f;
    for (int i = j + tid; i < m; i += TQ_THREADS) df::dot_acc(mjh[i], mjl[i], mjh[i], mjl[i], sh, sl);
    df::warp_sum(sh, sl);
    if (lane == 0) { red_h[warp] = sh; red_l[warp] = sl; }
    __syncthreads();
    if (tid == 0) {
      // the reflector's scalars in double-float too (an FP64 square root or
      // division is a long dependent chain on the FP64 pipe)
      float th = red_h[0], tl = red_l[0];
      for (int w = 1; w < TQ_THREADS / 32; ++w) df::add_to(th, tl, red_h[w], red_l[w]);
      const float xh = mjh[j], xl = mjl[j];
      float nh, nl;
      df::sqrt_df(th, tl, nh, nl);
      const float ah = (xh > 0.f) ? -nh : nh, al = (xh > 0.f) ? -nl : nl;
      float vh, vl, wh = nh, wl = nl, qh, ql;
      df::sub(xh, xl, ah, al, vh, vl);                                 // v0 = x0 - alpha
      df::add_to(wh, wl, fabsf(xh), xh < 0.f ? -xl : xl);               // nrm + |x0|
      df::mul(nh, nl, wh, wl, qh, ql);                                  // v^T v / 2
      sh_ah = ah;
      sh_al = al;
      if (qh > 0.f) {
        df::div_df(1.f, 0.f, qh, ql, sh_bh, sh_bl);                     // beta = 2 / v^T v
      } else {
        sh_bh = 0.f;
        sh_bl = 0.f;
      }
      mjh[j] = vh;
      mjl[j] = vl;
    }
    __syncthreads();
    const float bh = sh_bh, bl = sh_bl;
    if (bh != 0.f) {
      // one aligned 8-lane group per trailing column, TQ_THREADS / 8 columns per round
      for (int k0 = j + 1; k0 < c; k0 += TQ_THREADS / 8) {
        const int k = k0 + (tid >> 3), gl = tid & 7;
        const bool on = k < c;
        float* mkh = Mh + (on ? k : j) * ldm;
        float* mkl = Ml + (on ? k : j) * ldm;
        float dh = 0.f, dl = 0.f, eh = 0.f, el = 0.f;  // two chains for latency
        if (on) {
#pragma unroll
          for (int ii = 0; ii < 17; ii += 2) {  // rows j .. m - 1, m <= 136
            const int i = j + gl + 8 * ii, i2 = i + 8;
            if (i < m) df::dot_acc(mjh[i], mjl[i], mkh[i], mkl[i], dh, dl);
            if (ii + 1 < 17 && i2 < m) df::dot_acc(mjh[i2], mjl[i2], mkh[i2], mkl[i2], eh, el);
          }
          df::add_to(dh, dl, eh, el);
        }
        df::group8_sum(dh, dl);
        if (on) {
          float fh, fl;
          df::fast_two_sum(dh, dl, dh, dl);
          df::mul(bh, bl, dh, dl, fh, fl);
#pragma unroll
          for (int ii = 0; ii < 17; ++ii) {
            const int i = j + gl + 8 * ii;
            if (i < m) df::axpy_neg(fh, fl, mjh[i], mjl[i], mkh[i], mkl[i]);
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0) { mjh[j] = sh_ah; mjl[j] = sh_al; }
    __syncthreads();
  }
  double* Ro = R + (int64_t)tk.out_slot * c * c;
  for (int idx = tid; idx < c * c; idx += TQ_THREADS) {
    const int rr = idx / c, col = idx % c;
    Ro[idx] = (rr <= col && rr < steps) ? df::join(Mh[col * ldm + rr], Ml[col * ldm + rr]) : 0.0;
  }
}

// The merge of two c x c triangles R = qr([R1; R2]) of k_tsqr_merge (packed
// triangles, the j-th reflector touching row j of R1 and rows 0..j of R2) in
// double-float; FP64 in and out.
__global__ __launch_bounds__(TQ_THREADS) void k_tsqr_merge_df(const TsqrTask* __restrict__ tasks,
                                                              int c, double* __restrict__ R,
                                                              const NodeJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TsqrTask* tkp = tasks + blockIdx.x;
  if (jobs) {  // a level-wide launch over several operators' nodes
    const NodeJob& jb = jobs[blockIdx.x];
    tkp = jb.task;
    c = jb.c;
    R = jb.R;
  }
  const TsqrTask tk = *tkp;
  const int pk = c * (c + 1) / 2;
  float* Ah = reinterpret_cast<float*>(smem_raw);  // R1, packed upper
  float* Al = Ah + pk;
  float* Bh = Al + pk;                              // R2, packed upper
  float* Bl = Bh + pk;
  __shared__ float red_h[TQ_THREADS / 32], red_l[TQ_THREADS / 32];
  __shared__ float sh_ah, sh_al, sh_bh, sh_bl, sh_vh, sh_vl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* R1 = R + (int64_t)tk.slot[0] * c * c;
  const double* R2 = R + (int64_t)tk.slot[1] * c * c;
  for (int idx = tid; idx < c * c; idx += TQ_THREADS) {
    const int rr = idx / c, col = idx % c;
    if (rr <= col) {
      const int o = col * (col + 1) / 2 + rr;
      df::split(R1[idx], Ah[o], Al[o]);
      df::split(R2[idx], Bh[o], Bl[o]);
    }
  }
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    const int oj = j * (j + 1) / 2;  // rows 0..j of column j of R2
    float sh = 0.f, sl = 0.f;
    for (int i = tid; i <= j; i += TQ_THREADS) df::dot_acc(Bh[oj + i], Bl[oj + i], Bh[oj + i], Bl[oj + i], sh, sl);
    df::warp_sum(sh, sl);
    if (lane == 0) { red_h[warp] = sh; red_l[warp] = sl; }
    __syncthreads();
    if (tid == 0) {
      // the reflector's scalars in double-float (see k_tsqr_df)
      float th = red_h[0], tl = red_l[0];
      for (int w = 1; w < TQ_THREADS / 32; ++w) df::add_to(th, tl, red_h[w], red_l[w]);
      const float xh = Ah[oj + j], xl = Al[oj + j];
      float sh2, sl2, nh, nl;
      df::mul(xh, xl, xh, xl, sh2, sl2);
      df::add_to(sh2, sl2, th, tl);                                     // x0^2 + tail
      df::sqrt_df(sh2, sl2, nh, nl);
      const float ah = (xh > 0.f) ? -nh : nh, al = (xh > 0.f) ? -nl : nl;
      float vh, vl, wh = nh, wl = nl, qh, ql;
      df::sub(xh, xl, ah, al, vh, vl);                                 // v0 = x0 - alpha
      df::add_to(wh, wl, fabsf(xh), xh < 0.f ? -xl : xl);               // nrm + |x0|
      df::mul(nh, nl, wh, wl, qh, ql);                                  // v^T v / 2
      sh_ah = ah;
      sh_al = al;
      sh_vh = vh;
      sh_vl = vl;
      if (qh > 0.f) {
        df::div_df(1.f, 0.f, qh, ql, sh_bh, sh_bl);                     // beta = 2 / v^T v
      } else {
        sh_bh = 0.f;
        sh_bl = 0.f;
      }
    }
    __syncthreads();
    const float bh = sh_bh, bl = sh_bl, vh = sh_vh, vl = sh_vl;
    if (bh != 0.f) {
      // one aligned 8-lane group per trailing column, TQ_THREADS / 8 columns per round
      for (int k0 = j + 1; k0 < c; k0 += TQ_THREADS / 8) {
        const int k = k0 + (tid >> 3), gl = tid & 7;
        const bool on = k < c;
        const int kk = on ? k : j;
        const int ok = kk * (kk + 1) / 2;
        float dh = 0.f, dl = 0.f, eh = 0.f, el = 0.f;  // two chains for latency
        if (on) {
#pragma unroll
          for (int ii = 0; ii < 16; ii += 2) {  // rows 0 .. j, j < c <= 128
            const int i = gl + 8 * ii, i2 = i + 8;
            if (i <= j) df::dot_acc(Bh[oj + i], Bl[oj + i], Bh[ok + i], Bl[ok + i], dh, dl);
            if (i2 <= j) df::dot_acc(Bh[oj + i2], Bl[oj + i2], Bh[ok + i2], Bl[ok + i2], eh, el);
          }
          df::add_to(dh, dl, eh, el);
        }
        df::group8_sum(dh, dl);
        if (on) {
          // f = beta (dot + v0 A(j, k))
          df::dot_acc(vh, vl, Ah[ok + j], Al[ok + j], dh, dl);
          float fh, fl;
          df::fast_two_sum(dh, dl, dh, dl);
          df::mul(bh, bl, dh, dl, fh, fl);
#pragma unroll
          for (int ii = 0; ii < 16; ++ii) {
            const int i = gl + 8 * ii;
            if (i <= j) df::axpy_neg(fh, fl, Bh[oj + i], Bl[oj + i], Bh[ok + i], Bl[ok + i]);
          }
          if (gl == 0) df::axpy_neg(fh, fl, vh, vl, Ah[ok + j], Al[ok + j]);
        }
      }
    }
    __syncthreads();
    if (tid == 0 && bh != 0.f) { Ah[oj + j] = sh_ah; Al[oj + j] = sh_al; }
    __syncthreads();
  }
  double* Ro = R + (int64_t)tk.out_slot * c * c;
  for (int idx = tid; idx < c * c; idx += TQ_THREADS) {
    const int rr = idx / c, col = idx % c;
    const int o = col * (col + 1) / 2 + rr;
    Ro[idx] = (rr <= col) ? df::join(Ah[o], Al[o]) : 0.0;
  }
}
}  // namespace

void launch_jacobi_df(const int32_t* node_slot, int nnodes, const double* R, int c, double* W,
                      double* sigma, cudaStream_t st) {
  count_launches(1);
  const size_t smem = (size_t)3 * c * c * sizeof(float);
  static std::atomic<uint32_t> done{0};
  raise_smem_limit((const void*)k_jacobi_df, done);
  k_jacobi_df<<<nnodes, 512, smem, st>>>(node_slot, R, c, W, sigma, nullptr);
}

void launch_jacobi_df_jobs(const NodeJob* jobs, int njobs, int cmax, cudaStream_t st) {
  if (njobs <= 0) return;
  count_launches(1);
  const size_t smem = (size_t)3 * cmax * cmax * sizeof(float);
  static std::atomic<uint32_t> done{0};
  raise_smem_limit((const void*)k_jacobi_df, done);
  k_jacobi_df<<<njobs, 512, smem, st>>>(nullptr, nullptr, cmax, nullptr, nullptr, jobs);
}

void launch_tsqr_df(const TsqrTask* tasks, int ntasks, int merge, const double* P, int64_t ldp,
                    int c, double* R, cudaStream_t st) {
  count_launches(1);
  if (!merge) {
    const int ldm = kTsqrRows + 8;
    const size_t smem = (size_t)2 * ldm * c * sizeof(float);
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_tsqr_df, done);
    k_tsqr_df<<<ntasks, TQ_THREADS, smem, st>>>(tasks, P, ldp, c, R, ldm, nullptr);
  } else {
    const size_t smem = (size_t)2 * c * (c + 1) * sizeof(float);
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_tsqr_merge_df, done);
    k_tsqr_merge_df<<<ntasks, TQ_THREADS, smem, st>>>(tasks, c, R, nullptr);
  }
}

void launch_tsqr_df_jobs(const NodeJob* jobs, int njobs, int merge, int cmax, cudaStream_t st) {
  if (njobs <= 0) return;
  count_launches(1);
  if (!merge) {
    const int ldm = kTsqrRows + 8;
    const size_t smem = (size_t)2 * ldm * cmax * sizeof(float);
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_tsqr_df, done);
    k_tsqr_df<<<njobs, TQ_THREADS, smem, st>>>(nullptr, nullptr, 0, cmax, nullptr, ldm, jobs);
  } else {
    const size_t smem = (size_t)2 * cmax * (cmax + 1) * sizeof(float);
    static std::atomic<uint32_t> done{0};
    raise_smem_limit((const void*)k_tsqr_merge_df, done);
    k_tsqr_merge_df<<<njobs, TQ_THREADS, smem, st>>>(nullptr, cmax, nullptr, jobs);
  }
}

}  // namespace hm
