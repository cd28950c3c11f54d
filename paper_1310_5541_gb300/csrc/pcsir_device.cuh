// Device helpers shared by the pcSIR / SIR kernels: double-float arithmetic,
// fixed-point accumulation, ordered max of doubles, hashing, and the
// warp-cooperative patch likelihood of Eq. (likelihood).
#pragma once

#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "pcsir_internal.h"

namespace pcsir {

// ---------------------------------------------------------------------------
// Double-float ("float-float") arithmetic: a value is hi + lo with |lo| <=
// ulp(hi)/2.  Error-free transformations after Knuth (TwoSum) and Dekker
// (Fast2Sum), products through one FMA.  Every operation uses the _rn
// intrinsics so no contraction or reassociation can change the rounding.
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_from_double(double v) {
  float hi = __double2float_rn(v);
  float lo = __double2float_rn(__dsub_rn(v, (double)hi));
  return {hi, lo};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// exp of a double-float argument a <= 0, relative error about 1e-13.
// Range reduction a = k ln2 + r (|r| <= ln2/2) with ln2 as a double-float,
// then r' = r / 16, a degree-6 Taylor polynomial of exp(r') (the terms from
// r'^3 on are below 2^-24 of the result and are summed in float), four
// squarings, and the 2^k scale applied exactly to both parts.
__device__ __forceinline__ df df_exp_neg(df a) {
  if (a.hi < -87.0f) return {0.0f, 0.0f};
  const float LOG2E = 1.44269504088896341f;
  const df LN2 = {0.693147182464599609375f, -1.904654323148236017e-09f};
  float k = rintf(__fmul_rn(a.hi, LOG2E));
  df r = df_add(a, df_mul_f(LN2, -k));
  r.hi = __fmul_rn(r.hi, 0.0625f);
  r.lo = __fmul_rn(r.lo, 0.0625f);
  // 1 + r + r^2/2 in double-float, the rest in float
  df r2 = df_mul(r, r);
  r2.hi = __fmul_rn(r2.hi, 0.5f);
  r2.lo = __fmul_rn(r2.lo, 0.5f);
  float x = r.hi;
  float tail = x * x * x * (1.0f / 6.0f + x * (1.0f / 24.0f + x * (1.0f / 120.0f + x * (1.0f / 720.0f))));
  df p = df_add(r, r2);
  p = df_add_f(p, tail);
  p = df_add_f(p, 1.0f);
  p = df_mul(p, p);
  p = df_mul(p, p);
  p = df_mul(p, p);
  p = df_mul(p, p);
  // 2^k for k in [-126, 0] built from its exponent bits: one rounding per part, as ldexpf gives
  const float sc = __int_as_float(((int)k + 127) << 23);
  return {__fmul_rn(p.hi, sc), __fmul_rn(p.lo, sc)};
}

// phi(u) = u - log(1 + u) >= 0 for u > -1, computed without cancellation.
// For -1/2 <= u <= 1, with s = u / (2 + u) (|s| <= 1/3) and
// log(1+u) = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), u - 2 s = u s exactly,
// so phi = u s - 2 s^3 (1/3 + s^2/5 + ... + s^14/17); truncation error below
// 1e-9 relative.  Outside that range phi >= 0.19 and the direct difference is
// accurate with the fast logarithm (a few ulp of log(1 + u)); the fast form
// keeps the rare lanes outside the range from holding up their warp for a
// full-accuracy log1p (about 11% of SIR's likelihood time, measured).
__device__ __forceinline__ float phi_log1p(float u) {
  if (u >= -0.5f && u <= 1.0f) {
    float s = __fdividef(u, __fadd_rn(2.0f, u));  // 2 ulp, 2 + u in [1.5, 3]
    float s2 = s * s;
    float p = 1.0f / 17.0f;
    p = fmaf(p, s2, 1.0f / 15.0f);
    p = fmaf(p, s2, 1.0f / 13.0f);
    p = fmaf(p, s2, 1.0f / 11.0f);
    p = fmaf(p, s2, 1.0f / 9.0f);
    p = fmaf(p, s2, 1.0f / 7.0f);
    p = fmaf(p, s2, 1.0f / 5.0f);
    p = fmaf(p, s2, 1.0f / 3.0f);
    return fmaf(u, s, -2.0f * s * s2 * p);
  }
  return u - __logf(1.0f + u);
}

// Kahan-compensated accumulator in float.
struct kahan {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    float y = __fsub_rn(v, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
};

__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = df_add(v, w);
  }
  return v;
}

// ---------------------------------------------------------------------------
// Likelihood of one position, computed by a group of GS threads (a warp or
// several; Eq. object, Eq. likelihood).  The PSF factorises,
// lambda = I0 gx(px) gy(py) + bg, so the 2P one-dimensional factors are
// computed once in double-float (scratch in shared memory, 4P floats per
// group) and each of the P^2 pixels costs one double-float product.  For the
// Poisson term the difference d = lambda - z is rounded once to float and the
// term is -z phi(d / z).  Pixel terms are summed with Kahan compensation per
// thread, then in double-float across the group in a fixed order.
// All threads of the group must call this with the same arguments; every
// thread returns the result.
// ---------------------------------------------------------------------------
struct LikParams {
  int P;          // odd patch side
  int kind;       // PCSIR_LIK_*
  float bg;       // background
  df c2;          // 1 / (2 sigma^2) as double-float
  float inv2sxi2; // 1 / (2 sigma_xi^2)
};

// Conversions between floats and 64-bit fixed-point integers done with
// integer instructions: the hardware's 64-bit float <-> integer conversions
// run on this GPU's (slow) FP64 pipe.

// t * 2^32 truncated toward zero (|t| < 2^30; exact for |t| >= 2^-9)
__device__ __forceinline__ long long f2fix32(float t) {
  const unsigned b = __float_as_uint(t);
  const int e = (int)((b >> 23) & 0xffu);
  if (e == 0) return 0;
  const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = e - 118;  // t * 2^32 = m * 2^(e - 150 + 32)
  unsigned long long v;
  if (sh >= 0) v = sh < 39 ? (m << sh) : (1ull << 61);
  else v = sh > -24 ? (m >> -sh) : 0ull;
  return (b >> 31) ? -(long long)v : (long long)v;
}

// |d| truncated to 24 significant bits as a float; *back = its integer value
__device__ __forceinline__ float i64_trunc_float(long long d, long long* back) {
  if (d == 0) {
    *back = 0;
    return 0.0f;
  }
  const bool neg = d < 0;
  const unsigned long long a = neg ? 0ull - (unsigned long long)d : (unsigned long long)d;
  const int top = 63 - __clzll((long long)a);
  const int sh = top - 23;  // mantissa with its leading bit at position 23
  const unsigned long long mt = sh >= 0 ? a >> sh : a << (-sh);
  const unsigned long long tv = sh >= 0 ? mt << sh : a;
  *back = neg ? -(long long)tv : (long long)tv;
  return __uint_as_float((neg ? 0x80000000u : 0u) | ((unsigned)(top + 127) << 23) | (unsigned)(mt & 0x7fffffu));
}

// d * 2^-32 as a double-float (relative error below 2^-46)
__device__ __forceinline__ df fix32_to_df(long long d) {
  long long hb, lb;
  const float hi = i64_trunc_float(d, &hb);
  const float lo = i64_trunc_float(d - hb, &lb);
  const float sc = 2.3283064365386963e-10f;  // 2^-32
  return fast_two_sum(__fmul_rn(hi, sc), __fmul_rn(lo, sc));
}

// barrier over the GS threads of one group (GS = 32: the warp)
template <int GS>
__device__ __forceinline__ void group_sync(int group) {
  if (GS == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(GS) : "memory");
  }
}

// An evaluated position: coordinates and intensity as double-float, and the
// pixel nearest to it, (floor(x + 0.5), floor(y + 0.5)), computed exactly.
struct LikPos {
  df x, y, i0;
  int cx, cy;
};

// nearest pixel of a float coordinate without rounding x + 0.5: floor(x) and
// the fraction x - floor(x), which is exact except for x in (-1, 0), where
// its rounding cannot cross 1/2
__device__ __forceinline__ int nearest_pixel(float x) {
  const float f = floorf(x);
  return (int)f + (__fsub_rn(x, f) >= 0.5f ? 1 : 0);
}

__device__ __forceinline__ LikPos lik_pos(float x, float y, float i0) {
  LikPos q;
  q.x = {x, 0.0f};
  q.y = {y, 0.0f};
  q.i0 = {i0 > 0.0f ? i0 : 0.0f, 0.0f};
  q.cx = nearest_pixel(x);
  q.cy = nearest_pixel(y);
  return q;
}

__device__ __forceinline__ LikPos lik_pos(double x, double y, double i0) {
  LikPos q;
  q.x = df_from_double(x);
  q.y = df_from_double(y);
  q.i0 = df_from_double(i0 > 0.0 ? i0 : 0.0);
  q.cx = (int)floor(x + 0.5);
  q.cy = (int)floor(y + 0.5);
  return q;
}

// (integer pixel coordinate) - (double-float position), exactly rounded to a double-float
__device__ __forceinline__ df pixel_offset(int p, df x) {
  df d = two_sum((float)p, -x.hi);
  d.lo = __fsub_rn(d.lo, x.lo);
  return fast_two_sum(d.hi, d.lo);
}

// Log-likelihood as a double-float sum; bad if a pixel term was not a number
// (a non-finite image value).
struct LLSum {
  df sum;
  bool bad;
};

__device__ __forceinline__ double ll_to_double(LLSum s) {
  return s.bad ? -INFINITY : (double)s.sum.hi + (double)s.sum.lo;
}

template <int GS>
__device__ __forceinline__ LLSum group_loglik(const float* __restrict__ img, int W, int H, const LikPos& q,
                                               const LikParams& lp, float* __restrict__ scratch,
                                               int* __restrict__ red, int group, int gtid) {
  const int P = lp.P;
  const int R = P >> 1;
  const int cx = q.cx;
  const int cy = q.cy;
  const df I0 = q.i0;
  float* gxh = scratch;
  float* gxl = scratch + P;
  float* gyh = scratch + 2 * P;
  float* gyl = scratch + 3 * P;
  // one-dimensional factors: column j -> I0 * exp(-(px - x)^2 c2), row j -> exp(-(py - y)^2 c2)
  for (int j = gtid; j < 2 * P; j += GS) {
    const bool col = j < P;
    const int jj = col ? j : j - P;
    const df d = col ? pixel_offset(cx - R + jj, q.x) : pixel_offset(cy - R + jj, q.y);
    df e = df_mul(df_mul(d, d), lp.c2);
    e.hi = -e.hi;
    e.lo = -e.lo;
    df g = df_exp_neg(e);
    if (col) {
      g = df_mul(g, I0);
      gxh[jj] = g.hi;
      gxl[jj] = g.lo;
    } else {
      gyh[jj] = g.hi;
      gyl[jj] = g.lo;
    }
  }
  group_sync<GS>(group);
  kahan acc;
  bool bad = false;
  const int PP = P * P;
  // pixel p = r P + c, advanced by GS per iteration without integer division
  const int step_r = GS / P, step_c = GS - (GS / P) * P;
  int r = gtid / P, c = gtid - (gtid / P) * P;
  for (int p = gtid; p < PP; p += GS, r += step_r, c += step_c) {
    if (c >= P) {
      c -= P;
      ++r;
    }
    const int px = cx - R + c;
    const int py = cy - R + r;
    if (px < 0 || px >= W || py < 0 || py >= H) continue;
    const float z = __ldg(img + (size_t)py * W + px);
    const df prod = df_mul({gxh[c], gxl[c]}, {gyh[r], gyl[r]});  // I0 gx gy
    if (lp.kind == PCSIR_LIK_POISSON) {
      if (z > 0.0f) {
        // d = prod + (bg - z), rounded once
        const df s = two_sum(prod.hi, __fsub_rn(lp.bg, z));
        const float d = __fadd_rn(s.hi, __fadd_rn(s.lo, prod.lo));
        const float u = __fdividef(d, z);  // 2 ulp; z is a photon count, far inside the normal range
        // a NaN term (from a NaN pixel) makes the sum NaN, marked bad after the reduction
        acc.add(-z * phi_log1p(u));
      } else {
        const df lam = df_add_f(prod, lp.bg);
        bad |= (z != z);
        acc.add(-lam.hi);
        acc.add(-lam.lo);
      }
    } else {
      // e = z - lambda = (z - bg) - prod, rounded once
      const df s = two_sum(__fsub_rn(z, lp.bg), -prod.hi);
      const float e = __fadd_rn(s.hi, __fsub_rn(s.lo, prod.lo));
      acc.add(-(e * e) * lp.inv2sxi2);
    }
  }
  bad = __any_sync(0xffffffffu, bad);
  df tot = warp_sum_df(two_sum(acc.s, -acc.c));
  bad |= (tot.hi != tot.hi);  // a NaN Poisson term (the xor reduction gives every lane the same sum)
  if (GS > 32) {
    // warps' partial sums in a fixed order
    if ((gtid & 31) == 0) {
      red[2 * (gtid >> 5)] = __float_as_int(tot.hi);
      red[2 * (gtid >> 5) + 1] = bad ? 1 : 0;
      reinterpret_cast<float*>(red)[2 * (GS / 32) + (gtid >> 5)] = tot.lo;
    }
    group_sync<GS>(group);
    tot = {0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < GS / 32; ++k) {
      tot = df_add(tot, {__int_as_float(red[2 * k]), reinterpret_cast<float*>(red)[2 * (GS / 32) + k]});
      bad |= red[2 * k + 1] != 0;
    }
  }
  group_sync<GS>(group);  // scratch and red may be reused after this
  return {tot, bad};
}

// The Poisson likelihood at one position by an aligned group of GS lanes (GS = 8 or 16), every
// group of the warp at its own position: for small patches, where a whole warp per position
// leaves most lanes idle in the pixel loop and spends more on the per-position work.  All lanes of
// the warp call it together; a group with active == false takes no position (and returns zero).
// The same terms as group_loglik, summed over fewer lanes.  scratch: 4 P floats for this group.
template <int GS>
__device__ __forceinline__ LLSum subgroup_loglik(const float* __restrict__ img, int W, int H, const LikPos& q,
                                                 const LikParams& lp, float* __restrict__ scratch, bool active) {
  static_assert(GS == 8 || GS == 16, "sub-warp groups of 8 or 16 lanes");
  const int gtid = threadIdx.x & (GS - 1);
  const int P = active ? lp.P : 0;
  const int R = P >> 1;
  const int cx = q.cx, cy = q.cy;
  float* gxh = scratch;
  float* gxl = scratch + P;
  float* gyh = scratch + 2 * P;
  float* gyl = scratch + 3 * P;
  for (int j = gtid; j < 2 * P; j += GS) {
    const bool col = j < P;
    const int jj = col ? j : j - P;
    const df d = col ? pixel_offset(cx - R + jj, q.x) : pixel_offset(cy - R + jj, q.y);
    df e = df_mul(df_mul(d, d), lp.c2);
    e.hi = -e.hi;
    e.lo = -e.lo;
    df g = df_exp_neg(e);
    if (col) {
      g = df_mul(g, q.i0);
      gxh[jj] = g.hi;
      gxl[jj] = g.lo;
    } else {
      gyh[jj] = g.hi;
      gyl[jj] = g.lo;
    }
  }
  __syncwarp();
  kahan acc;
  bool bad = false;
  // pixel p = r P + c advanced by GS per iteration: GS = step_r P + step_c (step_c < P)
  const int step_r = P > 0 ? GS / P : 0, step_c = GS - step_r * P;
  int r = P > 0 ? gtid / P : 0, c = gtid - r * P;
  for (int p = gtid; p < P * P; p += GS, r += step_r, c += step_c) {
    if (c >= P) {
      c -= P;
      ++r;
    }
    const int px = cx - R + c;
    const int py = cy - R + r;
    if (px < 0 || px >= W || py < 0 || py >= H) continue;
    const float z = __ldg(img + (size_t)py * W + px);
    const df prod = df_mul({gxh[c], gxl[c]}, {gyh[r], gyl[r]});  // I0 gx gy
    if (z > 0.0f) {
      const df s2 = two_sum(prod.hi, __fsub_rn(lp.bg, z));
      const float d = __fadd_rn(s2.hi, __fadd_rn(s2.lo, prod.lo));
      acc.add(-z * phi_log1p(__fdividef(d, z)));  // a NaN term makes the sum NaN, marked bad below
    } else {
      const df lam = df_add_f(prod, lp.bg);
      bad |= (z != z);
      acc.add(-lam.hi);
      acc.add(-lam.lo);
    }
  }
  // the group's sum: xor shuffles over offsets below GS stay within the aligned group
  df tot = two_sum(acc.s, -acc.c);
#pragma unroll
  for (int o = GS / 2; o > 0; o >>= 1) {
    df w;
    w.hi = __shfl_xor_sync(0xffffffffu, tot.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, tot.lo, o);
    tot = df_add(tot, w);
  }
  const unsigned gmask = ((1u << GS) - 1u) << (threadIdx.x & 31 & ~(GS - 1));
  bad = (__ballot_sync(0xffffffffu, bad) & gmask) != 0u;
  bad |= (tot.hi != tot.hi);
  __syncwarp();  // scratch may be reused after this
  return {tot, bad};
}

// the warp version used per particle (SIR) and for stand-alone evaluations
__device__ __forceinline__ LLSum warp_loglik(const float* __restrict__ img, int W, int H, const LikPos& q,
                                             const LikParams& lp, float* __restrict__ scratch) {
  return group_loglik<32>(img, W, H, q, lp, scratch, nullptr, 0, threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// Order-preserving 64-bit encoding of doubles (for atomicMax).  0 encodes
// "nothing yet" and sorts below every real value.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ord_encode(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_decode(unsigned long long o) {
  unsigned long long b = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
  return __longlong_as_double((long long)b);
}

// ---------------------------------------------------------------------------
// Cell keys and hashing.  A cell (bx, by), |bx|,|by| < 2^30, is packed into a
// 64-bit key; all-ones never occurs and marks an empty hash slot.
// ---------------------------------------------------------------------------
constexpr unsigned long long EMPTY_KEY = 0xffffffffffffffffull;

__device__ __forceinline__ unsigned long long pack_key(int bx, int by) {
  return ((unsigned long long)(unsigned)(by + 0x40000000) << 32) | (unsigned)(bx + 0x40000000);
}
__device__ __forceinline__ int key_bx(unsigned long long k) { return (int)(unsigned)(k & 0xffffffffu) - 0x40000000; }
__device__ __forceinline__ int key_by(unsigned long long k) { return (int)(unsigned)(k >> 32) - 0x40000000; }

__device__ __forceinline__ unsigned hash_bits(unsigned long long k, int bits) {
  return (unsigned)((k * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

// Fixed-point scales of the centre-of-mass sums (see pcsir_internal.h).
constexpr double POS_SCALE = 2147483648.0;      // 2^31
constexpr double POS_INV = 1.0 / 2147483648.0;
constexpr double VAL_SCALE = 4194304.0;         // 2^22
constexpr double VAL_INV = 1.0 / 4194304.0;

// v * 2^shift rounded to the nearest integer (ties to even); exact whenever v * 2^shift is an
// integer.  v = t + f with t = trunc(v) and f = v - t, both exact: t 2^shift is an integer product
// and f 2^shift (|f| < 1, an exact scaling) is rounded to an int32.  |v| is clamped to 2^30 first
// (NaN to -2^30): every caller then finds the value outside its biased range and flags it, as it
// does any state component of 10^9 or more.
template <int SHIFT>
__device__ __forceinline__ long long fix_round(float v) {
  const float c = fminf(fmaxf(v, -1073741824.0f), 1073741824.0f);
  const float t = truncf(c);
  const int ti = __float2int_rz(t);
  const int fi = __float2int_rn(__fmul_rn(__fsub_rn(c, t), (float)(1ll << SHIFT)));
  return (long long)ti * (1ll << SHIFT) + (long long)fi;
}
__device__ __forceinline__ long long to_fixed(float v, float scale) {
  // the two scales used: 2^31 (positions) and 2^22 (other components)
  return scale > 4194304.0f ? fix_round<31>(v) : fix_round<22>(v);
}
__device__ __forceinline__ long long to_fixed(double v, double scale) {
  return __double2ll_rn(__dmul_rn(v, scale));
}

// Per-particle log-likelihoods kept as exact fixed-point integers (units of
// 2^-32, LLQ_NONE for "no weight"); max encoded for an unsigned atomicMax.
constexpr long long LLQ_NONE = LLONG_MIN;
constexpr long long LLQ_LIMIT = 1ll << 61;

__device__ __forceinline__ long long llq_of(LLSum s) {
  if (s.bad) return LLQ_NONE;
  const float lim = 5.0e8f;  // |ll| beyond this carries no usable weight
  if (!(fabsf(s.sum.hi) < lim)) return s.sum.hi > 0.0f ? f2fix32(lim) : -f2fix32(lim);
  return f2fix32(s.sum.hi) + f2fix32(s.sum.lo);
}
// caller-given log-weight in fixed point (non-finite or -inf: no weight)
__device__ __forceinline__ long long llq_of(double lw) {
  if (!(lw > -2.0e9 && lw < 2.0e9)) return lw == lw && lw > 0.0 ? LLQ_LIMIT : LLQ_NONE;
  return __double2ll_rn(lw * 4294967296.0);
}
__device__ __forceinline__ unsigned long long llq_enc(long long v) {
  return (unsigned long long)v ^ 0x8000000000000000ull;
}
__device__ __forceinline__ long long llq_dec(unsigned long long e) { return (long long)(e ^ 0x8000000000000000ull); }

// Per-particle weight w = exp(ll - max) <= 1 in double-float (relative error
// about 1e-13, so the integer weights below carry the scale's resolution),
// from the fixed-point log-likelihood and maximum without any FP64 operation,
// and its integer weight q = rint(w 2^sq), computed as the sum of the rounded
// scaled parts.  The weight reduction and the scan both call these, so both
// see identical q.
__device__ __forceinline__ df wtilde_q(long long llq, long long mq) {
  if (llq == LLQ_NONE) return {0.0f, 0.0f};
  long long d = llq - mq;  // <= 0; both lie within +-2^61
  if (d > 0) d = 0;
  return df_exp_neg(fix32_to_df(d));
}
// float -> int64 rounded to nearest, ties to even (the result of __float2ll_rn for |v| < 2^62),
// by integer instructions: the 64-bit conversion instruction runs on this GPU's slow FP64 pipe
__device__ __forceinline__ long long f2ll_rn_int(float v) {
  const unsigned b = __float_as_uint(v);
  const int e = (int)((b >> 23) & 0xffu);
  if (e == 0) return 0;  // zero or subnormal: |v| < 2^-126
  const unsigned m = (b & 0x7fffffu) | 0x800000u;
  const int sh = e - 150;  // |v| = m 2^sh
  unsigned long long r;
  if (sh >= 0) {
    r = (unsigned long long)m << (sh < 39 ? sh : 39);
  } else if (sh < -24) {
    r = 0ull;  // |v| < 1/2
  } else {
    const int k = -sh;
    const unsigned q = m >> k, rem = m & ((1u << k) - 1u), half = 1u << (k - 1);
    r = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
  }
  return (b >> 31) ? -(long long)r : (long long)r;
}
__device__ __forceinline__ long long q_of_wtilde(df w, int sq) {
  const float scale = __int_as_float((127 + sq) << 23);  // 2^sq, exact
  return f2ll_rn_int(__fmul_rn(w.hi, scale)) + f2ll_rn_int(__fmul_rn(w.lo, scale));
}

// Atomic OR of an error flag into the control block.
__device__ __forceinline__ void raise_flag(Control* ctl, unsigned f) { atomicOr(&ctl->err, f); }

// ---------------------------------------------------------------------------
// Likelihood surrogate: the input patch and the held-out selection.
// ---------------------------------------------------------------------------
constexpr int SUR_R = PCSIR_SUR_PATCH / 2;

// Nearest pixel (cx, cy) = (floor(x + 0.5), floor(y + 0.5)); false when the
// 21 x 21 patch around it leaves the image (or the position is not finite).
__device__ __forceinline__ bool sur_origin(double x, double y, int W, int H, int* cx, int* cy) {
  const double fx = floor(x + 0.5), fy = floor(y + 0.5);
  if (!(fx - SUR_R >= 0.0 && fx + SUR_R <= (double)(W - 1) && fy - SUR_R >= 0.0 && fy + SUR_R <= (double)(H - 1)))
    return false;
  *cx = (int)fx;
  *cy = (int)fy;
  return true;
}

// One output of the splitmix64 generator (Steele, Lea and Flood, 2014) whose
// state has just become x - 0x9E3779B97F4A7C15.
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Held-out threshold floor(max(frac, min_holdout / B) * 2^24) (2^24: every cell).
__device__ __forceinline__ unsigned sur_holdout_threshold(double frac, int min_holdout, unsigned B) {
  double f = frac;
  if (B > 0u) f = fmax(f, (double)min_holdout / (double)B);
  return f >= 1.0 ? (1u << 24) : (unsigned)floor(f * 16777216.0);
}

__device__ __forceinline__ bool sur_held(int bx, int by, unsigned long long salt, unsigned thr) {
  const unsigned long long key = (unsigned long long)(unsigned)bx | ((unsigned long long)(unsigned)by << 32);
  const unsigned long long h = splitmix64(key + salt * 0x9E3779B97F4A7C15ull);
  return (unsigned)(h >> 40) < thr;
}

}  // namespace pcsir
