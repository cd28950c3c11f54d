// Batched multi-target pcSIR in 3D (include/pcsir3.h): T independent targets,
// each its own Algorithm 2 filter over the state (x, y, z, vx, vy, vz, I0)
// with its own particle count, cell edges, PSF and patch, observed in one
// shared volume.  One step is a fixed sequence of kernels over all targets at
// once (capturable as one CUDA graph):
//   k_b3_prep       per-target anchors of the fixed-point sums
//   k_b3_prop_bin   propagate + 3D cell + exact centre-of-mass sums, cells keyed by target
//   k_b3_bins       dummies and their likelihood (one warp per occupied cell)
//   k_b3_weights    per-cell weights, integer weights, per-target sums
//   k_b3_tile_sums  per-(target, tile) sums of the integer weights
//   k_b3_scan       per-target scan of its tile sums, resampling map and results
//   k_b3_clear      occupied hash slots back to empty
//   k_b3_resample   per-(target, tile) systematic resampling and state gather
// No kernel waits for another block; every loop has a fixed bound.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pcsir_3d.cuh"

namespace pcsir {

constexpr int B3_MAX_TARGETS = 1023;
constexpr int B3_TILE = 4096;
constexpr int B3_RTHREADS = 512;
constexpr int B3_ITEMS = B3_TILE / B3_RTHREADS;  // 8
constexpr int B3_WTHREADS = 256;
constexpr float B3_LIM = 131070.0f;  // |cell index| < 2^17 - 1 per axis

struct Target3 {
  long long off, n;
  long long hq[3];  // cell edges in units of 2^-31 voxel
  float h[3];       // cell edges as float (the per-particle cell index)
  Lik3 lik;
  int sq;           // integer-weight scale bits, n 2^sq <= 2^61
  int tile0, ntiles;
};

struct TStats3 {  // per target, zeroed every step
  unsigned long long max_ll;
  double T_f, T2_f, est[NS3];
  long long T_int;
  long long anchor[4];
  unsigned long long dhi, dlo, uhi, ulo;
  float inv_delta;
  unsigned nbins;
};

struct B3Bufs {
  StepBuffers b;  // global cell table, occupied list, per-cell arrays, per-particle slots, tiles, control
  const Target3* tg;
  TStats3* ts;
  const long long* offs;   // [T + 1]
  const int* tile_target;  // [ntiles]
  unsigned long long* bin_key;
  pcsir3_result* res;      // [T]
  long long ntot;
  int T;
  int ntiles;
};

// cell key: target (10 bits) | bz + 2^17 | by + 2^17 | bx + 2^17 (18 bits each); |b| < 2^17 - 1
// keeps every field below all-ones, so the empty key never occurs
__device__ __forceinline__ unsigned long long b3_key(int t, int bx, int by, int bz) {
  return ((unsigned long long)t << 54) | ((unsigned long long)(unsigned)(bz + (1 << 17)) << 36) |
         ((unsigned long long)(unsigned)(by + (1 << 17)) << 18) | (unsigned long long)(unsigned)(bx + (1 << 17));
}
__device__ __forceinline__ int b3_t(unsigned long long k) { return (int)(k >> 54); }
__device__ __forceinline__ int b3_axis(unsigned long long k, int a) {
  return (int)((k >> (18 * a)) & 0x3ffffull) - (1 << 17);
}

// target owning particle i: offs[lo] <= i < offs[lo + 1] (offs in shared memory, T + 1 entries)
__device__ __forceinline__ int b3_target_of(const long long* offs, int T, long long i) {
  int lo = 0, hi = T;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (offs[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Anchors of the non-position components per target: the target's first
// particle's input values in fixed point (2^-22)
// ---------------------------------------------------------------------------
__global__ void k_b3_prep(B3Bufs B, const float* __restrict__ st) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B.T) return;
  const long long i = B.tg[t].off;
#pragma unroll
  for (int c = 0; c < 4; ++c) B.ts[t].anchor[c] = to_fixed(st[(3 + c) * B.ntot + i], 4194304.0f);
}

// ---------------------------------------------------------------------------
// Propagate + cell + centre-of-mass sums (Algorithm 2 per target, cells keyed
// by target), as k_prop_bin3 of the single-target step
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(P3_THREADS, 2)
k_b3_prop_bin(B3Bufs B, const float* __restrict__ st, const float* __restrict__ nz) {
  extern __shared__ __align__(16) unsigned char smem_b3[];
  Local3& tab = *reinterpret_cast<Local3*>(smem_b3);
  long long* offs = reinterpret_cast<long long*>(smem_b3 + sizeof(Local3));
  const StepBuffers& b = B.b;
  const long long N = B.ntot;
  float* __restrict__ prop = static_cast<float*>(b.prop);
  const size_t hcap = size_t(1) << b.hbits;
  for (int j = threadIdx.x; j < L3; j += blockDim.x) {
    tab.key[j] = EMPTY_KEY;
#pragma unroll
    for (int a = 0; a < NACC3; ++a) tab.acc[a][j] = 0u;
  }
  for (int t = threadIdx.x; t <= B.T; t += blockDim.x) offs[t] = B.offs[t];
  if (threadIdx.x == 0) {
    tab.fill = 0u;
    tab.hot = 0u;
  }
  __syncthreads();
  // each block takes a contiguous range of chunks: it meets the cells of one or two targets, which
  // its table holds, where a grid-stride order would show it every target's cells
  const long long nchunks = (N + P3_CHUNK - 1) / P3_CHUNK;
  const long long per_block = (nchunks + gridDim.x - 1) / gridDim.x;
  const long long c_begin = (long long)blockIdx.x * per_block;
  const long long c_end = c_begin + per_block < nchunks ? c_begin + per_block : nchunks;
  for (long long chunk = c_begin; chunk < c_end; ++chunk) {
    const long long base = chunk * P3_CHUNK;
    float v[P3_PER_THREAD][NS3];
    // each particle is summed into its cell as soon as the cell is found; ls: the cell's local
    // slot, -3 - its global slot (table full), or -2 (no particle)
    int ls[P3_PER_THREAD];
    bool flag = false;  // this thread filled the table or brought a cell's count to the flush mark
    int t = b3_target_of(offs, B.T, base + threadIdx.x < N ? base + threadIdx.x : N - 1);
#pragma unroll
    for (int k = 0; k < P3_PER_THREAD; ++k) {
      const long long i = base + (long long)k * P3_THREADS + threadIdx.x;
      ls[k] = -2;
      if (i >= N) continue;
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        v[k][p] = __fadd_rn(__fadd_rn(st[p * N + i], st[(3 + p) * N + i]), nz[p * N + i]);
        v[k][3 + p] = __fadd_rn(st[(3 + p) * N + i], nz[(3 + p) * N + i]);
      }
      v[k][6] = __fadd_rn(st[6 * N + i], nz[6 * N + i]);
#pragma unroll
      for (int c = 0; c < NS3; ++c) prop[c * N + i] = v[k][c];
    }
#pragma unroll
    for (int k = 0; k < P3_PER_THREAD; ++k) {
      const long long i = base + (long long)k * P3_THREADS + threadIdx.x;
      if (i >= N) continue;
      while (t + 1 < B.T && offs[t + 1] <= i) ++t;
      const Target3& T_ = B.tg[t];
      bool ok = true;
      float f[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        f[p] = floorf(__fdiv_rn(__fadd_rn(v[k][p], 0.5f), T_.h[p]));
        ok &= fabsf(f[p]) < B3_LIM;
      }
#pragma unroll
      for (int c = 0; c < NS3; ++c) ok &= fabsf(v[k][c]) < 1.0e9f;
      if (!ok) {
        raise_flag(b.ctl, PCSIR_DERR_RANGE);
        f[0] = f[1] = f[2] = 0.0f;
        v[k][0] = v[k][1] = v[k][2] = 0.0f;
      }
      const unsigned long long key = b3_key(t, (int)f[0], (int)f[1], (int)f[2]);
      bool created;
      int s = local_insert3(tab, key, created, flag);
      if (created) tab.gslot[s] = global_insert3(b, key);
      const TStats3& S_ = B.ts[t];
      long long bv[NS3];
#pragma unroll
      for (int p = 0; p < 3; ++p)
        bv[p] = to_fixed(v[k][p], 2147483648.0f) - (long long)(int)f[p] * T_.hq[p] + P3_POS_BIAS;
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[3 + c] = to_fixed(v[k][3 + c], 4194304.0f) - S_.anchor[c] + P3_VAL_BIAS;
      bool bad = false;
#pragma unroll
      for (int c = 0; c < NS3; ++c) bad |= (bv[c] < 0 || bv[c] >= P3_LIMIT);
      if (bad) {
        raise_flag(b.ctl, PCSIR_DERR_RANGE);
#pragma unroll
        for (int c = 0; c < NS3; ++c) bv[c] = bias3(c);
      }
      if (s >= 0) {
        if (atomicAdd(&tab.acc[0][s], 1u) + 1u == P3_HOT_AT) flag = true;
#pragma unroll
        for (int c = 0; c < NS3; ++c) {
          atomicAdd(&tab.acc[1 + 2 * c][s], (unsigned)(bv[c] & P3_PIECE_MASK));
          atomicAdd(&tab.acc[2 + 2 * c][s], (unsigned)(bv[c] >> P3_PIECE_BITS));
        }
      } else {
        const unsigned g = global_insert3(b, key);
        atomicAdd(&b.hcnt[g], 1u);
#pragma unroll
        for (int c = 0; c < NS3; ++c)
          atomicAdd((unsigned long long*)&b.hsum[c * hcap + g], (unsigned long long)(bv[c] - bias3(c)));
        s = -3 - (int)g;
      }
      ls[k] = s;
    }
    // flushed after this chunk when some thread filled the table or raised a cell to the flush
    // mark: every thread learns it from the barrier itself, never from the table's counters,
    // which the next chunk's inserts may already change
    const bool flush = __syncthreads_or(flag) != 0;
#pragma unroll
    for (int k = 0; k < P3_PER_THREAD; ++k) {
      if (ls[k] == -2) continue;
      const long long i = base + (long long)k * P3_THREADS + threadIdx.x;
      b.pslot[i] = ls[k] >= 0 ? tab.gslot[ls[k]] : (unsigned)(-3 - ls[k]);
    }
    if (flush) local_flush3(tab, b, tab.fill >= L3_CAP);  // read before the flush's first barrier
  }
  local_flush3(tab, b, false);
}


// ---------------------------------------------------------------------------
// Dummies (the members' mean state) and their likelihood with the target's
// PSF and patch: one warp per occupied cell
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(B3_WTHREADS) k_b3_bins(B3Bufs B, const float* __restrict__ vol, int W, int H, int D) {
  constexpr int NW = B3_WTHREADS / 32;
  __shared__ float scratch[NW][2 * (3 * MAXP3)];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const StepBuffers& b = B.b;
  const unsigned nb = b.ctl->nocc;
  const size_t hcap = size_t(1) << b.hbits;
  const int64_t bs = b.bin_stride;
  for (unsigned bi = blockIdx.x * NW + w; bi < nb; bi += gridDim.x * NW) {
    const unsigned g = b.occ[bi];
    const unsigned long long key = b.hkey[g];
    const int t = b3_t(key);
    const Target3& T_ = B.tg[t];
    const TStats3& S_ = B.ts[t];
    const double dn = (double)b.hcnt[g];
    const double rdn = 1.0 / dn;  // one FP64 division per cell (GB300's FP64 rate is low)
    double mean[NS3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
      mean[p] = ((double)((long long)b3_axis(key, p) * T_.hq[p]) + (double)b.hsum[p * hcap + g] * rdn) * POS_INV;
#pragma unroll
    for (int c = 3; c < NS3; ++c) mean[c] = ((double)S_.anchor[c - 3] + (double)b.hsum[c * hcap + g] * rdn) * VAL_INV;
    double ll =
        ll_to_double(warp_loglik3(vol, W, H, D, pos3(mean[0], mean[1], mean[2], mean[6]), T_.lik, scratch[w]));
    if (!isfinite(ll)) {
      if (lane == 0) raise_flag(b.ctl, PCSIR_DERR_NONFINITE);
      ll = -INFINITY;
    }
    if (lane == 0) {
      B.bin_key[bi] = key;
      b.bin_cnt[bi] = b.hcnt[g];
#pragma unroll
      for (int c = 0; c < NS3; ++c) b.dummy[c * bs + bi] = mean[c];
      b.bin_ll[bi] = ll;
      if (ll > -INFINITY) atomicMax(&B.ts[t].max_ll, ord_encode(ll));
      atomicAdd(&B.ts[t].nbins, 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// Per cell: w~ = exp(ll - max_t), integer weight q = rint(w~ 2^sq_t), and the
// target's normaliser, sum of squares, posterior-mean sums (from the exact
// fixed-point sums) and integer total
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(B3_WTHREADS) k_b3_weights(B3Bufs B) {
  const StepBuffers& b = B.b;
  const unsigned nb = b.ctl->nocc;
  const size_t hcap = size_t(1) << b.hbits;
  for (unsigned bi = blockIdx.x * blockDim.x + threadIdx.x; bi < nb; bi += gridDim.x * blockDim.x) {
    const unsigned g = b.occ[bi];
    const unsigned long long key = B.bin_key[bi];
    const int t = b3_t(key);
    const Target3& T_ = B.tg[t];
    TStats3& S_ = B.ts[t];
    const double m = ord_decode(*(volatile unsigned long long*)&S_.max_ll);
    const double ll = b.bin_ll[bi];
    const double wt = (ll == -INFINITY) ? 0.0 : exp(ll - m);
    const long long q = __double2ll_rn(ldexp(wt, T_.sq));
    b.hq[g] = q;
    const unsigned n = b.bin_cnt[bi];
    atomicAdd(&S_.T_f, n * wt);
    atomicAdd(&S_.T2_f, n * wt * wt);
    atomicAdd((unsigned long long*)&S_.T_int, (unsigned long long)((long long)n * q));
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const double sp = ((double)((long long)b3_axis(key, p) * T_.hq[p]) * n + (double)b.hsum[p * hcap + g]) * POS_INV;
      atomicAdd(&S_.est[p], wt * sp);
    }
#pragma unroll
    for (int c = 3; c < NS3; ++c) {
      const double sc = ((double)S_.anchor[c - 3] * n + (double)b.hsum[c * hcap + g]) * VAL_INV;
      atomicAdd(&S_.est[c], wt * sc);
    }
  }
}

// per-(target, tile) sums of the integer weights of the tile's particles
__global__ void __launch_bounds__(B3_RTHREADS) k_b3_tile_sums(B3Bufs B) {
  __shared__ long long red[B3_RTHREADS / 32];
  const int item = blockIdx.x;
  const int t = B.tile_target[item];
  const Target3& T_ = B.tg[t];
  const long long base = T_.off + (long long)(item - T_.tile0) * B3_TILE;
  const long long end = T_.off + T_.n;
  long long s = 0;
  for (int j = threadIdx.x; j < B3_TILE; j += blockDim.x) {
    const long long i = base + j;
    if (i < end) s += B.b.hq[B.b.pslot[i]];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tot = 0;
    for (int k = 0; k < B3_RTHREADS / 32; ++k) tot += red[k];
    B.b.tile_sum[item] = tot;
  }
}

// one warp per target: exclusive scan of its tile sums, the 64.64 resampling map
// (Delta = T / n, U0 = u0 Delta) and the target's results
__global__ void __launch_bounds__(B3_WTHREADS) k_b3_scan(B3Bufs B, const double* __restrict__ u0s) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= B.T) return;
  const Target3& T_ = B.tg[t];
  TStats3& S_ = B.ts[t];
  long long e = 0;
  for (int k0 = 0; k0 < T_.ntiles; k0 += 32) {
    const int k = k0 + lane;
    const long long v = k < T_.ntiles ? B.b.tile_sum[T_.tile0 + k] : 0ll;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (k < T_.ntiles) B.b.tile_excl[T_.tile0 + k] = e + inc - v;
    e += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (lane != 0) return;
  const unsigned long long Tq = (unsigned long long)e;
  const unsigned long long n = (unsigned long long)T_.n;
  S_.dhi = Tq / n;
  S_.dlo = (unsigned long long)(((unsigned __int128)(Tq % n) << 64) / n);
  const double dd = (double)S_.dhi + (double)S_.dlo * 5.421010862427522e-20;
  S_.inv_delta = dd > 0.0 ? (float)(1.0 / dd) : 0.0f;
  double uf = u0s[t] * 18446744073709551616.0;
  if (!(uf >= 0.0)) uf = 0.0;
  const unsigned long long u0f = uf >= 18446744073709549568.0 ? 18446744073709549568ull : __double2ull_rz(uf);
  const unsigned __int128 tot = (unsigned __int128)u0f * S_.dhi + (((unsigned __int128)u0f * S_.dlo) >> 64);
  S_.uhi = (unsigned long long)(tot >> 64);
  S_.ulo = (unsigned long long)tot;
  pcsir3_result& r = B.res[t];
  const double Tf = S_.T_f;
  for (int c = 0; c < NS3; ++c) r.estimate[c] = S_.est[c] / Tf;
  r.ess = Tf * Tf / S_.T2_f;
  r.max_loglik = ord_decode(S_.max_ll);
  r.sum_wtilde = Tf;
  r.n_particles = T_.n;
  r.n_bins = S_.nbins;
  r.kind = 1;
  r.device_error = Tq == 0ull ? PCSIR_DERR_ZEROSUM : 0;
  if (Tq == 0ull) raise_flag(B.b.ctl, PCSIR_DERR_ZEROSUM);
}

// the step's occupied hash slots back to empty (after the weights have been read)
__global__ void k_b3_clear(B3Bufs B) {
  const StepBuffers& b = B.b;
  const unsigned nb = b.ctl->nocc;
  const size_t hcap = size_t(1) << b.hbits;
  for (unsigned bi = blockIdx.x * blockDim.x + threadIdx.x; bi < nb; bi += gridDim.x * blockDim.x) {
    const unsigned g = b.occ[bi];
    b.hkey[g] = EMPTY_KEY;
    b.hcnt[g] = 0u;
#pragma unroll
    for (int c = 0; c < NS3; ++c) b.hsum[c * hcap + g] = 0;
  }
}

// ---------------------------------------------------------------------------
// Systematic resampling per (target, tile): the tile's inclusive cumulative
// integer weights in shared memory; output i of the target takes the particle
// j with C_{j-1} <= U_i < C_j, U_i = i Delta + U0 in 64.64 fixed point, i.e.
// the number of C_j <= floor(U_i) (exact: the C_j are integers)
// ---------------------------------------------------------------------------
// integer part of i Delta + U0
__device__ __forceinline__ long long b3_u(const TStats3& S, long long i) {
  const unsigned long long ui = (unsigned long long)i;
  const unsigned long long plo = ui * S.dlo;
  const unsigned long long phi = __umul64hi(ui, S.dlo);
  const unsigned long long s = plo + S.ulo;
  return (long long)(ui * S.dhi + S.uhi + phi + (s < plo ? 1ull : 0ull));
}

// first output i in [0, n] with U_i >= C: a float guess of (C - U0) / Delta corrected exactly
__device__ long long b3_first_out(const TStats3& S, long long C, long long n) {
  if (C <= 0) return 0;
  if (S.dhi == 0ull && S.dlo == 0ull) return n;
  long long back;
  const float cf = i64_trunc_float(C - (long long)S.uhi, &back);
  const float xf = __fmul_rn(cf, S.inv_delta);
  long long i = xf <= 0.0f ? 0 : (xf >= (float)n ? n : (long long)__float2int_rn(xf));
  int guard = 0;
  while (i > 0 && b3_u(S, i - 1) >= C && guard++ < 256) --i;
  while (i < n && b3_u(S, i) < C && guard++ < 512) ++i;
  return i;
}

// number of the tile's C_j <= u, over Cs padded as j + j / 16 (fixed 12-step search)
__device__ __forceinline__ int b3_search(const long long* __restrict__ Cs, long long u) {
  int pa = 0;
#pragma unroll
  for (int step = B3_TILE / 2; step > 0; step >>= 1)
    if (Cs[pa + (step - 1) + ((step - 1) >> 4)] <= u) pa += step + (step >> 4);
  return pa - pa / 17;
}

__global__ void __launch_bounds__(B3_RTHREADS) k_b3_resample(B3Bufs B, float* __restrict__ out) {
  __shared__ long long Cs[B3_TILE + B3_TILE / 16];
  __shared__ long long wtot[B3_RTHREADS / 32];
  __shared__ long long s_lo, s_hi;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const StepBuffers& b = B.b;
  const long long Ntot = B.ntot;
  const float* __restrict__ prop = static_cast<const float*>(b.prop);
  const int item = blockIdx.x;
  const int t = B.tile_target[item];
  const Target3& T_ = B.tg[t];
  const TStats3& S_ = B.ts[t];
  const long long lbase = (long long)(item - T_.tile0) * B3_TILE;
  const long long n = T_.n;
  const int cnt = (int)((n - lbase) < B3_TILE ? (n - lbase) : B3_TILE);
  const long long excl = b.tile_excl[item];
  long long loc[B3_ITEMS];
  long long run = 0;
#pragma unroll
  for (int k = 0; k < B3_ITEMS; ++k) {
    const int j = tid * B3_ITEMS + k;
    const long long q = j < cnt ? b.hq[b.pslot[T_.off + lbase + j]] : 0ll;
    if (b.qout != nullptr && j < cnt) b.qout[T_.off + lbase + j] = q;
    run += q;
    loc[k] = run;
  }
  long long inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wtot[w] = inc;
  __syncthreads();
  long long woff = 0, agg = 0;
#pragma unroll
  for (int j = 0; j < B3_RTHREADS / 32; ++j) {
    const long long v = wtot[j];
    if (j < w) woff += v;
    agg += v;
  }
  const long long texcl = woff + inc - run;
  // entries past the tile's last particle compare above every U_i
#pragma unroll
  for (int k = 0; k < B3_ITEMS; ++k) {
    const int jj = tid * B3_ITEMS + k;
    Cs[jj + (jj >> 4)] = jj < cnt ? excl + texcl + loc[k] : LLONG_MAX;
  }
  if (tid == 0) s_lo = b3_first_out(S_, excl, n);
  if (tid == 32) s_hi = (lbase + cnt >= n) ? n : b3_first_out(S_, excl + agg, n);
  __syncthreads();
  const long long lo = s_lo, hi = s_hi;
  const bool zero_sum = (S_.dhi == 0ull && S_.dlo == 0ull);
  for (long long i0 = lo + tid; i0 < hi; i0 += 2 * B3_RTHREADS) {
    long long src[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const long long i = i0 + (long long)j * B3_RTHREADS;
      int a = 0;
      if (i < hi && !zero_sum) {
        a = b3_search(Cs, b3_u(S_, i));
        a = a < cnt ? a : cnt - 1;
      }
      // all weights zero: no distribution to sample, every particle kept
      src[j] = zero_sum ? T_.off + i : T_.off + lbase + a;
      if (b.anc != nullptr && i < hi) b.anc[T_.off + i] = (int32_t)(src[j] - T_.off);
    }
    float v[2][NS3];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const bool has = i0 + (long long)j * B3_RTHREADS < hi;
#pragma unroll
      for (int d = 0; d < NS3; ++d) v[j][d] = has ? prop[d * Ntot + src[j]] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const long long i = i0 + (long long)j * B3_RTHREADS;
      if (i < hi) {
#pragma unroll
        for (int d = 0; d < NS3; ++d) out[d * Ntot + T_.off + i] = v[j][d];
      }
    }
  }
}

}  // namespace pcsir

// ---------------------------------------------------------------------------
// Host API
// ---------------------------------------------------------------------------
using namespace pcsir;

struct pcsir3_batch {
  int T = 0;
  long long ntot = 0;
  int ntiles = 0;
  int num_sms = 0;
  int pb_grid = 0;
  int keep = 0;
  B3Bufs B{};
  std::vector<void*> allocs;
  pcsir3_result* host_res = nullptr;
  std::string err = "no error";
  bool failed = false;
  bool stepped = false;
};

namespace {

template <typename X>
bool b3alloc(pcsir3_batch* c, X** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(X) + 16) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->allocs.push_back(q);
  *p = static_cast<X*>(q);
  return true;
}

void b3free(pcsir3_batch* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->host_res) cudaFreeHost(c->host_res);
  c->host_res = nullptr;
}

constexpr size_t B3_PB_SMEM = sizeof(Local3) + sizeof(long long) * (B3_MAX_TARGETS + 1);

}  // namespace

extern "C" {

const char* pcsir3_batch_last_error(pcsir3_batch* c) { return c ? c->err.c_str() : "NULL batch"; }

pcsir_status pcsir3_batch_create(const pcsir3_target* targets, int32_t T, int32_t keep, pcsir3_batch** out) {
  if (!out) return PCSIR_EINVAL;
  *out = nullptr;
  if (!targets || T < 1 || T > B3_MAX_TARGETS) return PCSIR_EINVAL;
  if (keep & ~(PCSIR_KEEP_ANCESTORS | PCSIR_KEEP_QWEIGHTS)) return PCSIR_EINVAL;
  std::vector<Target3> tg(T);
  long long ntot = 0;
  int ntiles = 0;
  for (int t = 0; t < T; ++t) {
    const pcsir3_target& x = targets[t];
    const double hh[3] = {x.hx, x.hy, x.hz};
    for (double h : hh)
      if (!(h > 0.0 && h <= MAX_H)) return PCSIR_EINVAL;
    if (x.n_particles < 1 || !(x.psf_sigma_xy > 0.0) || !(x.psf_sigma_z > 0.0) || !(x.bg > 0.0) ||
        !std::isfinite(x.psf_sigma_xy) || !std::isfinite(x.psf_sigma_z) || !std::isfinite(x.bg) ||
        x.patch_xy < 1 || x.patch_xy > MAXP3 || (x.patch_xy & 1) == 0 || x.patch_z < 1 || x.patch_z > MAXP3 ||
        (x.patch_z & 1) == 0)
      return PCSIR_EINVAL;
    Target3& g = tg[t];
    g.off = ntot;
    g.n = x.n_particles;
    for (int p = 0; p < 3; ++p) {
      g.h[p] = (float)hh[p];
      g.hq[p] = llrint((double)g.h[p] * 2147483648.0);
    }
    g.lik.Pxy = x.patch_xy;
    g.lik.Pz = x.patch_z;
    g.lik.bg = (float)x.bg;
    const double cxy = 1.0 / (2.0 * x.psf_sigma_xy * x.psf_sigma_xy);
    const double cz = 1.0 / (2.0 * x.psf_sigma_z * x.psf_sigma_z);
    g.lik.c2xy = {(float)cxy, (float)(cxy - (double)(float)cxy)};
    g.lik.c2z = {(float)cz, (float)(cz - (double)(float)cz)};
    g.sq = weight_scale_bits(x.n_particles);
    g.tile0 = ntiles;
    g.ntiles = (int)((x.n_particles + B3_TILE - 1) / B3_TILE);
    ntot += x.n_particles;
    ntiles += g.ntiles;
  }
  if (ntot > MAX_PARTICLES) return PCSIR_ERANGE;
  pcsir3_batch* c = new (std::nothrow) pcsir3_batch();
  if (!c) return PCSIR_ENOMEM;
  c->T = T;
  c->ntot = ntot;
  c->ntiles = ntiles;
  c->keep = keep;
  int hbits = 10;
  while ((1ll << hbits) < 2 * ntot) ++hbits;
  const size_t hcap = size_t(1) << hbits;
  B3Bufs& B = c->B;
  StepBuffers& b = B.b;
  b.hbits = hbits;
  b.bin_stride = ntot;
  b.max_tiles = ntiles;
  B.T = T;
  B.ntot = ntot;
  B.ntiles = ntiles;
  Target3* dtg = nullptr;
  long long* doffs = nullptr;
  int* dtile = nullptr;
  float* prop = nullptr;
  bool ok = b3alloc(c, &b.hkey, hcap) && b3alloc(c, &b.hcnt, hcap) && b3alloc(c, &b.hsum, (size_t)NS3 * hcap) &&
            b3alloc(c, &b.hq, hcap) && b3alloc(c, &b.occ, (size_t)ntot) && b3alloc(c, &b.bin_cnt, (size_t)ntot) &&
            b3alloc(c, &b.bin_ll, (size_t)ntot) && b3alloc(c, &b.dummy, (size_t)NS3 * ntot) &&
            b3alloc(c, &B.bin_key, (size_t)ntot) && b3alloc(c, &b.pslot, (size_t)ntot) &&
            b3alloc(c, &prop, (size_t)NS3 * ntot) && b3alloc(c, &b.tile_sum, (size_t)ntiles) &&
            b3alloc(c, &b.tile_excl, (size_t)ntiles) && b3alloc(c, &b.ctl, 1) && b3alloc(c, &dtg, (size_t)T) &&
            b3alloc(c, &B.ts, (size_t)T) && b3alloc(c, &doffs, (size_t)T + 1) && b3alloc(c, &dtile, (size_t)ntiles) &&
            b3alloc(c, &B.res, (size_t)T);
  if (ok && (keep & PCSIR_KEEP_ANCESTORS)) ok = b3alloc(c, &b.anc, (size_t)ntot);
  if (ok && (keep & PCSIR_KEEP_QWEIGHTS)) ok = b3alloc(c, &b.qout, (size_t)ntot);
  if (!ok) {
    b3free(c);
    delete c;
    return PCSIR_ENOMEM;
  }
  b.prop = prop;
  B.tg = dtg;
  B.offs = doffs;
  B.tile_target = dtile;
  std::vector<long long> offs(T + 1);
  for (int t = 0; t < T; ++t) offs[t] = tg[t].off;
  offs[T] = ntot;
  std::vector<int> tile_target(ntiles);
  for (int t = 0; t < T; ++t)
    for (int k = 0; k < tg[t].ntiles; ++k) tile_target[tg[t].tile0 + k] = t;
  int dev = 0, per_sm = 0;
  cudaError_t e = cudaMemcpy(dtg, tg.data(), sizeof(Target3) * T, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(doffs, offs.data(), sizeof(long long) * (T + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dtile, tile_target.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b.hkey, 0xff, hcap * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(b.hcnt, 0, hcap * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(b.hsum, 0, (size_t)NS3 * hcap * sizeof(long long));
  if (e == cudaSuccess) e = cudaMallocHost(&c->host_res, sizeof(pcsir3_result) * T);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_b3_prop_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B3_PB_SMEM);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b3_prop_bin, P3_THREADS, B3_PB_SMEM);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    b3free(c);
    delete c;
    return e == cudaErrorMemoryAllocation ? PCSIR_ENOMEM : PCSIR_ECUDA;
  }
  std::memset(c->host_res, 0, sizeof(pcsir3_result) * T);
  c->pb_grid = c->num_sms * std::max(1, per_sm);
  *out = c;
  return PCSIR_OK;
}

pcsir_status pcsir3_batch_destroy(pcsir3_batch* c) {
  if (!c) return PCSIR_OK;
  cudaDeviceSynchronize();
  b3free(c);
  delete c;
  return PCSIR_OK;
}

}  // extern "C"

extern "C" {

pcsir_status pcsir3_batched_step(pcsir3_batch* c, float* state, const float* volume, int32_t W, int32_t H, int32_t D,
                                 const float* noise, const double* u0, void* stream) {
  if (!c) return PCSIR_EINVAL;
  if (c->failed) return PCSIR_ESTATE;
  if (!state || !volume || !noise || !u0 || W < 1 || H < 1 || D < 1) {
    c->err = "NULL pointer or empty volume";
    return PCSIR_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const B3Bufs& B = c->B;
  const int T = c->T;
  const long long N = c->ntot;
  cudaError_t e = cudaMemsetAsync(B.b.ctl, 0, sizeof(Control), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.ts, 0, sizeof(TStats3) * T, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.res, 0, sizeof(pcsir3_result) * T, s);
  if (e == cudaSuccess) {
    k_b3_prep<<<(T + 255) / 256, 256, 0, s>>>(B, state);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const long long nchunks = (N + P3_CHUNK - 1) / P3_CHUNK;
    const int grid = (int)std::min<long long>(nchunks, (long long)c->pb_grid);
    k_b3_prop_bin<<<grid, P3_THREADS, B3_PB_SMEM, s>>>(B, state, noise);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_b3_bins<<<c->num_sms * 8, B3_WTHREADS, 0, s>>>(B, volume, W, H, D);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_b3_weights<<<c->num_sms * 4, B3_WTHREADS, 0, s>>>(B);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_b3_tile_sums<<<c->ntiles, B3_RTHREADS, 0, s>>>(B);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_b3_scan<<<(T + B3_WTHREADS / 32 - 1) / (B3_WTHREADS / 32), B3_WTHREADS, 0, s>>>(B, u0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_b3_clear<<<c->num_sms * 4, 256, 0, s>>>(B);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_b3_resample<<<c->ntiles, B3_RTHREADS, 0, s>>>(B, state);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->host_res, B.res, sizeof(pcsir3_result) * T, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->err = std::string("batched 3D step: ") + cudaGetErrorString(e);
    c->failed = true;
    return PCSIR_ECUDA;
  }
  c->stepped = true;
  return PCSIR_OK;
}

pcsir_status pcsir3_batch_results(pcsir3_batch* c, pcsir3_result* out, int32_t T, int32_t* device_error) {
  if (!c || !out || T != c->T) return PCSIR_EINVAL;
  // the step's copy of the results to page-locked memory is asynchronous: wait for it
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return PCSIR_ECUDA;
  }
  std::memcpy(out, c->host_res, sizeof(pcsir3_result) * T);
  if (device_error) {
    Control ctl;
    if (cudaMemcpy(&ctl, c->B.b.ctl, sizeof(ctl), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return PCSIR_ECUDA;
    }
    *device_error = (int32_t)ctl.err;
  }
  return PCSIR_OK;
}

pcsir_status pcsir3_batch_get_outputs(pcsir3_batch* c, pcsir3_batch_outputs* o) {
  if (!c || !o) return PCSIR_EINVAL;
  if (!c->stepped) return PCSIR_ESTATE;
  Control ctl;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&ctl, c->B.b.ctl, sizeof(ctl), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PCSIR_ECUDA;
  }
  const StepBuffers& b = c->B.b;
  std::memset(o, 0, sizeof(*o));
  o->n_total = c->ntot;
  o->n_bins = ctl.nocc;
  o->bin_stride = b.bin_stride;
  o->prop_state = static_cast<const float*>(b.prop);
  o->bin_key = reinterpret_cast<const uint64_t*>(c->B.bin_key);
  o->bin_count = b.bin_cnt;
  o->dummy = b.dummy;
  o->bin_loglik = b.bin_ll;
  o->particle_slot = b.pslot;
  o->ancestor = b.anc;
  o->qweight = reinterpret_cast<const int64_t*>(b.qout);
  return PCSIR_OK;
}

}  // extern "C"
