// Process noise drawn in the propagation kernel (pcsir_step_philox): the
// nearly-constant-velocity transition's five Gaussian increments (Section
// 5.1) from a counter-based generator, so that no noise array is read.
//
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC 2011): counter
// (i mod 2^32, i div 2^32, frame, j), j = 0, 1, for particle i, and the
// 64-bit seed as the key; ten rounds of the two published multipliers with
// the Weyl key schedule.  The first six of the eight outputs give three
// Box-Muller pairs, of which five normals are used.
//
// Every floating-point step is an IEEE single-precision operation with one
// rounding (explicit _rn intrinsics, never contracted into a fused
// multiply-add) or an exact bit operation, so that a CPU implementation of
// the same steps gets the same numbers: log u = e ln 2 + 2 atanh(s) with
// s = (m - 1)/(m + 1), m in [sqrt(1/2), sqrt(2)), by the series to s^9; the
// angle 2 pi u reduced exactly to a quadrant and a fraction folded to
// [0, 1/2], whose sine and cosine come from their Taylor series to x^9 and
// x^10.
#pragma once

#include <cstdint>

namespace pcsir {

struct NoiseGen {
  unsigned long long seed;
  unsigned int frame;
  float q[5];  // standard deviations of the five increments, rounded to float
};

__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // each 32 x 32 -> 64-bit product in one wide multiply, both halves from its register pair
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c[0];
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// series coefficients: the double constants rounded to float once
constexpr float NG_L3 = (float)(1.0 / 3.0), NG_L5 = (float)(1.0 / 5.0), NG_L7 = (float)(1.0 / 7.0),
                NG_L9 = (float)(1.0 / 9.0);
constexpr float NG_LN2 = (float)0.6931471805599453, NG_SQRT2 = (float)1.4142135623730951;
constexpr float NG_S3 = (float)(-1.0 / 6.0), NG_S5 = (float)(1.0 / 120.0), NG_S7 = (float)(-1.0 / 5040.0),
                NG_S9 = (float)(1.0 / 362880.0);
constexpr float NG_C2 = (float)(-1.0 / 2.0), NG_C4 = (float)(1.0 / 24.0), NG_C6 = (float)(-1.0 / 720.0),
                NG_C8 = (float)(1.0 / 40320.0), NG_C10 = (float)(-1.0 / 3628800.0);
constexpr float NG_HALF_PI = (float)(3.141592653589793 / 2.0);

// log u for u in (0, 1]
__device__ __forceinline__ float ng_log(float u) {
  const uint32_t bits = __float_as_uint(u);
  int e = (int)(bits >> 23) - 127;
  float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
  if (m > NG_SQRT2) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float p = NG_L9;
  p = __fadd_rn(__fmul_rn(p, s2), NG_L7);
  p = __fadd_rn(__fmul_rn(p, s2), NG_L5);
  p = __fadd_rn(__fmul_rn(p, s2), NG_L3);
  float a = __fmul_rn(s, s2);
  a = __fmul_rn(a, p);
  a = __fadd_rn(s, a);
  return __fadd_rn(__fmul_rn((float)e, NG_LN2), __fadd_rn(a, a));
}

// cos and sin of 2 pi u for u in [0, 1)
__device__ __forceinline__ void ng_sincos_turn(float u, float* c, float* s) {
  const float q4 = __fmul_rn(u, 4.0f);
  const float quad = floorf(q4);
  const float f = __fsub_rn(q4, quad);
  const bool fold = f > 0.5f;
  const float g = fold ? __fsub_rn(1.0f, f) : f;
  const float x = __fmul_rn(g, NG_HALF_PI);
  const float x2 = __fmul_rn(x, x);
  float p = NG_S9;
  p = __fadd_rn(__fmul_rn(p, x2), NG_S7);
  p = __fadd_rn(__fmul_rn(p, x2), NG_S5);
  p = __fadd_rn(__fmul_rn(p, x2), NG_S3);
  const float sn = __fadd_rn(x, __fmul_rn(__fmul_rn(x, x2), p));
  float cc = NG_C10;
  cc = __fadd_rn(__fmul_rn(cc, x2), NG_C8);
  cc = __fadd_rn(__fmul_rn(cc, x2), NG_C6);
  cc = __fadd_rn(__fmul_rn(cc, x2), NG_C4);
  cc = __fadd_rn(__fmul_rn(cc, x2), NG_C2);
  const float cs = __fadd_rn(1.0f, __fmul_rn(x2, cc));
  const float ca = fold ? sn : cs, sa = fold ? cs : sn;  // the angle within its quadrant
  const int qi = (int)quad;
  *c = qi == 0 ? ca : (qi == 1 ? -sa : (qi == 2 ? -ca : sa));
  *s = qi == 0 ? sa : (qi == 1 ? ca : (qi == 2 ? -sa : -ca));
}

__device__ __forceinline__ void ng_box_muller(uint32_t ra, uint32_t rb, float* z0, float* z1) {
  const float u1 = __fmul_rn((float)((ra >> 8) + 1u), 5.9604644775390625e-8f);  // (0, 1]
  const float u2 = __fmul_rn((float)(rb >> 8), 5.9604644775390625e-8f);         // [0, 1)
  const float rad = __fsqrt_rn(__fmul_rn(ng_log(u1), -2.0f));
  float c, s;
  ng_sincos_turn(u2, &c, &s);
  *z0 = __fmul_rn(rad, c);
  *z1 = __fmul_rn(rad, s);
}

// the five noise increments of particle i: q_d z_d
__device__ __forceinline__ void ng_noise5(const NoiseGen& ng, long long i, float e[5]) {
  const uint32_t k0 = (uint32_t)ng.seed, k1 = (uint32_t)(ng.seed >> 32);
  uint32_t a[4] = {(uint32_t)i, (uint32_t)((unsigned long long)i >> 32), ng.frame, 0u};
  uint32_t b[4] = {a[0], a[1], ng.frame, 1u};
  philox10(a, k0, k1);
  philox10(b, k0, k1);
  float z[6];
  ng_box_muller(a[0], a[1], &z[0], &z[1]);
  ng_box_muller(a[2], a[3], &z[2], &z[3]);
  ng_box_muller(b[0], b[1], &z[4], &z[5]);
#pragma unroll
  for (int d = 0; d < 5; ++d) e[d] = __fmul_rn(ng.q[d], z[d]);
}

}  // namespace pcsir
