// Device code shared by the single-target and the batched 3D steps: cell keys,
// the warp likelihood of an anisotropic Gaussian PSF over a voxel patch
// (Eq. object, Eq. likelihood; Poisson term), and the block-private cell table
// with exact fixed-point centre-of-mass sums flushed to the global table.
#pragma once

#include "pcsir3.h"
#include "pcsir_device.cuh"

namespace pcsir {

constexpr int NS3 = 7;
constexpr int NACC3 = 1 + 2 * NS3;  // count, (lo, hi) per component
constexpr int P3_THREADS = 512;
constexpr int P3_PER_THREAD = 2;  // two particles per thread: 64 registers, two blocks per SM
constexpr int P3_CHUNK = P3_THREADS * P3_PER_THREAD;
constexpr int L3_BITS = 10;
constexpr int L3 = 1 << L3_BITS;
constexpr unsigned L3_CAP = 768;
constexpr int P3_PIECE_BITS = 18;
constexpr unsigned P3_PIECE_MASK = (1u << P3_PIECE_BITS) - 1u;
// a slot's 32-bit counters hold the pieces (< 2^18) of at most 2^14 particles; the table is
// flushed after any chunk that leaves some slot at 2^14 - P3_CHUNK particles or more
constexpr unsigned P3_HOT_AT = (1u << 14) - (unsigned)P3_CHUNK;
constexpr long long P3_POS_BIAS = 1ll << 33;
constexpr long long P3_VAL_BIAS = 1ll << 34;
constexpr long long P3_LIMIT = 1ll << 36;
constexpr int MAXP3 = 63;

// cell key: 21 bits per axis (indices biased by 2^20); the top bit stays 0, so
// the all-ones empty key never occurs
__device__ __forceinline__ unsigned long long pack_key3(int bx, int by, int bz) {
  return (unsigned long long)(unsigned)(bx + (1 << 20)) | ((unsigned long long)(unsigned)(by + (1 << 20)) << 21) |
         ((unsigned long long)(unsigned)(bz + (1 << 20)) << 42);
}
__device__ __forceinline__ int key3(unsigned long long k, int axis) {
  return (int)((k >> (21 * axis)) & 0x1fffffull) - (1 << 20);
}

// ---------------------------------------------------------------------------
// Likelihood of one position by a warp (Eq. object with an anisotropic
// Gaussian PSF, Eq. likelihood; Poisson term).  The PSF factorises into
// three one-dimensional factor tables (double-float, in shared memory); each
// voxel costs two double-float products.
// ---------------------------------------------------------------------------
struct Lik3 {
  int Pxy, Pz;
  float bg;
  df c2xy, c2z;  // 1 / (2 sigma^2)
};

struct Pos3 {
  df x, y, z, i0;
  int cx, cy, cz;
};

__device__ __forceinline__ Pos3 pos3(float x, float y, float z, float i0) {
  Pos3 q;
  q.x = {x, 0.0f};
  q.y = {y, 0.0f};
  q.z = {z, 0.0f};
  q.i0 = {i0 > 0.0f ? i0 : 0.0f, 0.0f};
  q.cx = nearest_pixel(x);
  q.cy = nearest_pixel(y);
  q.cz = nearest_pixel(z);
  return q;
}
__device__ __forceinline__ Pos3 pos3(double x, double y, double z, double i0) {
  Pos3 q;
  q.x = df_from_double(x);
  q.y = df_from_double(y);
  q.z = df_from_double(z);
  q.i0 = df_from_double(i0 > 0.0 ? i0 : 0.0);
  q.cx = (int)floor(x + 0.5);
  q.cy = (int)floor(y + 0.5);
  q.cz = (int)floor(z + 0.5);
  return q;
}

// scratch: 2 (2 Pxy + Pz) floats per warp
static __device__ LLSum warp_loglik3(const float* __restrict__ vol, int W, int H, int D, const Pos3& q, const Lik3& lp,
                              float* __restrict__ scratch) {
  const int lane = threadIdx.x & 31;
  const int Pxy = lp.Pxy, Pz = lp.Pz;
  const int Rxy = Pxy >> 1, Rz = Pz >> 1;
  const int nf = 2 * Pxy + Pz;
  float* fh = scratch;
  float* fl = scratch + nf;
  // factors: [0, Pxy) x (times I0), [Pxy, 2 Pxy) y, [2 Pxy, nf) z
  for (int j = lane; j < nf; j += 32) {
    df d, c2;
    if (j < Pxy) {
      d = pixel_offset(q.cx - Rxy + j, q.x);
      c2 = lp.c2xy;
    } else if (j < 2 * Pxy) {
      d = pixel_offset(q.cy - Rxy + (j - Pxy), q.y);
      c2 = lp.c2xy;
    } else {
      d = pixel_offset(q.cz - Rz + (j - 2 * Pxy), q.z);
      c2 = lp.c2z;
    }
    df e = df_mul(df_mul(d, d), c2);
    e.hi = -e.hi;
    e.lo = -e.lo;
    df g = df_exp_neg(e);
    if (j < Pxy) g = df_mul(g, q.i0);
    fh[j] = g.hi;
    fl[j] = g.lo;
  }
  __syncwarp();
  kahan acc;
  bool bad = false;
  const int PP = Pxy * Pxy;
  const int total = PP * Pz;
  // voxel p = (s Pxy + r) Pxy + c, advanced by 32 per iteration in mixed radix (no integer division
  // in the loop): 32 = step_s PP + step_r Pxy + step_c
  const int step_s = 32 / PP, step_r = (32 - step_s * PP) / Pxy, step_c = 32 - step_s * PP - step_r * Pxy;
  int s = lane / PP, r = (lane - s * PP) / Pxy, c = lane - s * PP - r * Pxy;
  for (int p = lane; p < total; p += 32, c += step_c, r += step_r, s += step_s) {
    if (c >= Pxy) {
      c -= Pxy;
      ++r;
    }
    if (r >= Pxy) {
      r -= Pxy;
      ++s;
    }
    const int px = q.cx - Rxy + c, py = q.cy - Rxy + r, pz = q.cz - Rz + s;
    if (px < 0 || px >= W || py < 0 || py >= H || pz < 0 || pz >= D) continue;
    const float z = __ldg(vol + ((size_t)pz * H + py) * W + px);
    const df gxy = df_mul({fh[c], fl[c]}, {fh[Pxy + r], fl[Pxy + r]});
    const df prod = df_mul(gxy, {fh[2 * Pxy + s], fl[2 * Pxy + s]});  // I0 gx gy gz
    if (z > 0.0f) {
      const df sm = two_sum(prod.hi, __fsub_rn(lp.bg, z));
      const float d = __fadd_rn(sm.hi, __fadd_rn(sm.lo, prod.lo));
      const float u = __fdividef(d, z);
      acc.add(-z * phi_log1p(u));  // a NaN term makes the sum NaN, marked bad below
    } else {
      const df lam = df_add_f(prod, lp.bg);
      bad |= (z != z);
      acc.add(-lam.hi);
      acc.add(-lam.lo);
    }
  }
  bad = __any_sync(0xffffffffu, bad);
  const df tot = warp_sum_df(two_sum(acc.s, -acc.c));
  bad |= (tot.hi != tot.hi);
  __syncwarp();
  return {tot, bad};
}

// ---------------------------------------------------------------------------
// Global table
// ---------------------------------------------------------------------------
static __device__ unsigned global_insert3(const StepBuffers& b, unsigned long long key) {
  const unsigned mask = (1u << b.hbits) - 1u;
  unsigned h = hash_bits(key, b.hbits);
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const unsigned long long k = *(volatile unsigned long long*)&b.hkey[h];
    if (k == key) return h;
    if (k == EMPTY_KEY) {
      const unsigned long long old = atomicCAS(&b.hkey[h], EMPTY_KEY, key);
      if (old == EMPTY_KEY) {
        const unsigned idx = atomicAdd(&b.ctl->nocc, 1u);
        b.occ[idx] = h;
        return h;
      }
      if (old == key) return h;
    }
    h = (h + 1u) & mask;
  }
  raise_flag(b.ctl, PCSIR_DERR_RANGE);
  return 0;
}

struct Local3 {
  unsigned long long key[L3];
  unsigned int acc[NACC3][L3];
  unsigned int gslot[L3];
  unsigned int fill;
  unsigned int hot;  // some slot may reach 2^14 particles within the next chunk: flush
};

// filled: set when this call's claim brought the table to its capacity (the table is emptied
// after the chunk)
__device__ __forceinline__ int local_insert3(Local3& t, unsigned long long key, bool& created, bool& filled) {
  created = false;
  unsigned h = hash_bits(key, L3_BITS);
  for (int probe = 0; probe < L3; ++probe) {
    const unsigned long long k = ((volatile unsigned long long*)t.key)[h];
    if (k == key) return (int)h;
    if (k == EMPTY_KEY) {
      const unsigned f = atomicAdd(&t.fill, 1u);
      if (f + 1u >= L3_CAP) filled = true;
      if (f >= L3_CAP) return -1;
      const unsigned long long old = atomicCAS(&t.key[h], EMPTY_KEY, key);
      if (old == EMPTY_KEY) {
        created = true;
        return (int)h;
      }
      if (old == key) return (int)h;
    }
    h = (h + 1u) & (L3 - 1u);
  }
  return -1;
}

__device__ __forceinline__ long long bias3(int c) { return c < 3 ? P3_POS_BIAS : P3_VAL_BIAS; }

static __device__ void local_flush3(Local3& t, const StepBuffers& b, bool clear_keys) {
  const size_t hcap = size_t(1) << b.hbits;
  for (unsigned j = threadIdx.x; j < (unsigned)L3; j += blockDim.x) {
    if (t.key[j] == EMPTY_KEY) continue;
    const unsigned cnt = t.acc[0][j];
    if (cnt != 0u) {
      const unsigned g = t.gslot[j];
      atomicAdd(&b.hcnt[g], cnt);
#pragma unroll
      for (int c = 0; c < NS3; ++c) {
        const long long sum = (long long)t.acc[1 + 2 * c][j] + ((long long)t.acc[2 + 2 * c][j] << P3_PIECE_BITS) -
                              (long long)cnt * bias3(c);
        atomicAdd((unsigned long long*)&b.hsum[c * hcap + g], (unsigned long long)sum);
      }
#pragma unroll
      for (int a = 0; a < NACC3; ++a) t.acc[a][j] = 0u;
    }
    if (clear_keys) t.key[j] = EMPTY_KEY;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (clear_keys) t.fill = 0u;
    t.hot = 0u;
  }
  __syncthreads();
}

}  // namespace pcsir
