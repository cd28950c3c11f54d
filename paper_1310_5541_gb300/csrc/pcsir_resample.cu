// Systematic resampling (Algorithm 1/2 resampling step) as one pass over the
// particles: integer weights, single-pass decoupled look-back prefix scan,
// and the gather of the selected propagated states into the caller's buffer.
//
// Weights enter as integers q_i = rint(exp(ll_i - max) 2^sq), so the
// cumulative sums C_j are exact and independent of the summation order.
// Output i takes the first particle j with C_j > U_i, where
// U_i = (i + u0) T / N and T = C_{N-1}; U_i is evaluated in 64.64 fixed point
// as i * Delta + U0 with Delta = T / N and U0 = u0 * Delta, and only its
// integer part is compared with the integer C_j, which decides C_j > U_i
// exactly.  Each tile of particles owns the outputs whose U falls between its
// exclusive and inclusive prefixes, so every output is written exactly once.
#include <cmath>

#include "pcsir_device.cuh"

namespace pcsir {

constexpr unsigned long long ST_AGG = 1ull << 62;
constexpr unsigned long long ST_PREFIX = 1ull << 63;
constexpr unsigned long long ST_VAL = (1ull << 62) - 1ull;
constexpr int LOOKBACK_SPIN_LIMIT = 1 << 22;

struct Map64 {
  unsigned long long dhi, dlo, uhi, ulo;
  double dd, ud;
};

// integer part of i * Delta + U0
__device__ __forceinline__ long long u_int(const Map64& mp, long long i) {
  const unsigned __int128 lo = (unsigned __int128)(unsigned long long)i * mp.dlo + mp.ulo;
  return (long long)((unsigned long long)i * mp.dhi + mp.uhi + (unsigned long long)(lo >> 64));
}

// first output index i in [0, N] with U_i >= C
__device__ long long first_out(const Map64& mp, long long C, long long N) {
  if (C <= 0) return 0;
  double x = ((double)C - mp.ud) / mp.dd;
  long long i = (long long)ceil(x);
  if (i < 0) i = 0;
  if (i > N) i = N;
  int guard = 0;
  while (i > 0 && u_int(mp, i - 1) >= C && guard++ < 64) --i;
  while (i < N && u_int(mp, i) < C && guard++ < 128) ++i;
  return i;
}

__device__ __forceinline__ int pad_idx(int j) { return j + (j >> 4); }

// Exclusive prefix of a tile by decoupled look-back, done by one warp: each
// lane reads one predecessor's status word (waiting, with a bound, until it
// is published), the nearest predecessor holding an inclusive prefix ends the
// walk, and the aggregates in between are summed.
__device__ __forceinline__ long long lookback_warp(unsigned long long* st, long long tile, Control* ctl) {
  const int lane = threadIdx.x & 31;
  long long excl = 0;
  long long j = tile - 1;
  while (j >= 0) {
    const long long idx = j - lane;
    unsigned long long s = ST_PREFIX;  // before tile 0: an inclusive prefix of 0
    if (idx >= 0) {
      int spins = 0;
      while (true) {
        s = *(volatile unsigned long long*)&st[idx];
        if (s != 0ull) break;
        if (++spins > LOOKBACK_SPIN_LIMIT) {
          atomicOr(&ctl->err, (unsigned)PCSIR_DERR_TIMEOUT);
          s = ST_PREFIX;
          break;
        }
        __nanosleep(32);
      }
    }
    const unsigned pmask = __ballot_sync(0xffffffffu, (s & ST_PREFIX) != 0ull);
    const int first = pmask ? __ffs(pmask) - 1 : 32;
    long long c = lane <= first ? (long long)(s & ST_VAL) : 0ll;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    excl += c;
    if (pmask) break;
    j -= 32;
  }
  return excl;
}

template <typename T, int WSRC>
__global__ void __launch_bounds__(SCAN_THREADS, 4)
k_scan_resample(StepBuffers b, const double* __restrict__ lsrc, T* __restrict__ out, int64_t N, double u0,
                int sq, int keep) {
  __shared__ long long Cs[SCAN_TILE + SCAN_TILE / 16];
  __shared__ long long wtot[SCAN_THREADS / 32];
  __shared__ unsigned s_tile;
  __shared__ long long s_excl, s_lo, s_hi;
  __shared__ Map64 s_map;
  Control* ctl = b.ctl;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(&ctl->tile_ticket, 1u);
    // Delta = T / N and U0 = u0 Delta in 64.64 fixed point
    const unsigned long long T = (unsigned long long)*(volatile long long*)&ctl->T_int;
    const unsigned long long n = (unsigned long long)N;
    Map64 mp;
    mp.dhi = T / n;
    const unsigned long long rem = T % n;
    mp.dlo = (unsigned long long)(((unsigned __int128)rem << 64) / n);
    double uf = u0 * 18446744073709551616.0;
    if (!(uf >= 0.0)) uf = 0.0;
    const unsigned long long u0f = uf >= 18446744073709549568.0 ? 18446744073709549568ull : __double2ull_rz(uf);
    const unsigned __int128 ph = (unsigned __int128)u0f * mp.dhi;
    const unsigned __int128 pl = ((unsigned __int128)u0f * mp.dlo) >> 64;
    const unsigned __int128 tot = ph + pl;
    mp.uhi = (unsigned long long)(tot >> 64);
    mp.ulo = (unsigned long long)tot;
    mp.dd = (double)mp.dhi + (double)mp.dlo * 5.421010862427522e-20;
    mp.ud = (double)mp.uhi + (double)mp.ulo * 5.421010862427522e-20;
    s_map = mp;
  }
  __syncthreads();
  const unsigned tile = s_tile;
  const int64_t base = (int64_t)tile * SCAN_TILE;
  const int cnt = (int)((N - base) < SCAN_TILE ? (N - base) : SCAN_TILE);
  const double m = ord_decode(ctl->max_ll);
  const size_t hcap = size_t(1) << b.hbits;

  // 1. integer weights of the tile into padded shared memory; four
  //    consecutive particles per thread and load, all loads issued together
  if (WSRC == WSRC_BINS) {
    const bool vec = cnt == SCAN_TILE && (base % 4 == 0);
    unsigned g[SCAN_ITEMS];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS / 4; ++k) {
      const int j0 = k * (4 * SCAN_THREADS) + 4 * tid;
      if (vec) {
        const uint4 q4 = *reinterpret_cast<const uint4*>(b.pslot + base + j0);
        g[4 * k] = q4.x;
        g[4 * k + 1] = q4.y;
        g[4 * k + 2] = q4.z;
        g[4 * k + 3] = q4.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) g[4 * k + e] = (j0 + e < cnt) ? b.pslot[base + j0 + e] : 0xffffffffu;
      }
    }
    long long q[SCAN_ITEMS];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) q[k] = g[k] != 0xffffffffu ? b.hq[g[k]] : 0ll;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS / 4; ++k) {
      const int j0 = k * (4 * SCAN_THREADS) + 4 * tid;
#pragma unroll
      for (int e = 0; e < 4; ++e) Cs[pad_idx(j0 + e)] = q[4 * k + e];
    }
  } else {
#pragma unroll 4
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      const int j = k * SCAN_THREADS + tid;
      long long q = 0;
      if (j < cnt) q = q_of_wtilde(wtilde_df(lsrc[base + j], m), sq);
      Cs[pad_idx(j)] = q;
    }
  }
  __syncthreads();
  // 2. each thread scans its ITEMS consecutive weights
  long long run = 0;
  long long loc[SCAN_ITEMS];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    run += Cs[pad_idx(tid * SCAN_ITEMS + k)];
    loc[k] = run;
  }
  // 3. exclusive scan of the thread totals across the block
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
  for (int j = 0; j < SCAN_THREADS / 32; ++j) {
    const long long t = wtot[j];
    if (j < w) woff += t;
    agg += t;
  }
  const long long texcl = woff + inc - run;
  // 4. decoupled look-back for the tile's exclusive prefix
  if (w == 0) {
    unsigned long long* st = b.tile_status;
    if (lane == 0) atomicExch(&st[tile], (tile == 0 ? ST_PREFIX : ST_AGG) | (unsigned long long)agg);
    long long excl = 0;
    if (tile > 0) excl = lookback_warp(st, (long long)tile, ctl);
    if (lane == 0) {
      if (tile > 0) atomicExch(&st[tile], ST_PREFIX | (unsigned long long)(excl + agg));
      s_excl = excl;
      s_lo = first_out(s_map, excl, N);
      s_hi = (base + cnt >= N) ? N : first_out(s_map, excl + agg, N);
    }
  }
  __syncthreads();
  const long long excl = s_excl;
  // 5. inclusive cumulative weights C_j of the tile
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) Cs[pad_idx(tid * SCAN_ITEMS + k)] = excl + texcl + loc[k];
  __syncthreads();
  // 6. outputs owned by the tile: ancestor = first j with C_j > U_i, found from
  //    a proportional guess and a short walk (binary search if the walk is long)
  const Map64 mp = s_map;
  const T* __restrict__ prop = static_cast<const T*>(b.prop);
  const long long lo = s_lo, hi = s_hi;
  const long long nout = hi - lo;
  const bool zero_sum = (mp.dhi == 0ull && mp.dlo == 0ull);
  for (long long i = lo + tid; i < hi; i += SCAN_THREADS) {
    const long long U = u_int(mp, i);
    int a = (int)(((i - lo) * (long long)cnt) / (nout > 0 ? nout : 1));
    if (a >= cnt) a = cnt - 1;
    int steps = 0;
    while (a < cnt - 1 && Cs[pad_idx(a)] <= U && steps < 8) {
      ++a;
      ++steps;
    }
    while (a > 0 && Cs[pad_idx(a - 1)] > U && steps < 8) {
      --a;
      ++steps;
    }
    if (steps >= 8) {
      int l = 0, r = cnt;
      while (l < r) {
        const int mid = (l + r) >> 1;
        if (Cs[pad_idx(mid)] > U) r = mid;
        else l = mid + 1;
      }
      a = l < cnt ? l : cnt - 1;
    }
    // all weights zero (Delta = 0): no distribution to sample, keep every particle
    const int64_t anc = zero_sum ? (int64_t)i : base + a;
    if (out != nullptr) {
#pragma unroll
      for (int d = 0; d < 5; ++d) out[d * N + i] = prop[d * N + anc];
    }
    if (keep & PCSIR_KEEP_ANCESTORS) b.anc[i] = (int32_t)anc;
  }
  // 7. optional per-particle outputs of the tile
  if (keep & (PCSIR_KEEP_WEIGHTS | PCSIR_KEEP_PARTICLE_BIN)) {
    const double Tf = *(volatile double*)&ctl->T_f;
    for (int j = tid; j < cnt; j += SCAN_THREADS) {
      const int64_t i = base + j;
      if (WSRC == WSRC_BINS) {
        const unsigned g = b.pslot[i];
        if (keep & PCSIR_KEEP_WEIGHTS) b.wout[i] = b.hw[g] / Tf;
        if (keep & PCSIR_KEEP_PARTICLE_BIN) b.pbin[i] = b.hrank[g];
      } else if (keep & PCSIR_KEEP_WEIGHTS) {
        const double ll = lsrc[i];
        b.wout[i] = (ll == -INFINITY ? 0.0 : exp(ll - m)) / Tf;
      }
    }
  }
  // 8. pcSIR: return the occupied hash slots to empty for the next step
  if (WSRC == WSRC_BINS) {
    const unsigned B = ctl->nocc;
    for (unsigned bi = tile * SCAN_THREADS + tid; bi < B; bi += gridDim.x * SCAN_THREADS) {
      const unsigned g = b.occ[bi];
      b.hkey[g] = EMPTY_KEY;
      b.hcnt[g] = 0u;
#pragma unroll
      for (int d = 0; d < 5; ++d) b.hsum[d * hcap + g] = 0;
    }
  }
  // 9. the last tile to finish publishes the step's device error flags
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&ctl->tiles_done, 1u) == gridDim.x - 1) {
      __threadfence();
      b.dres->device_error = (int32_t)(*(volatile unsigned*)&ctl->err);
    }
  }
}

template <typename T>
static cudaError_t resample_launch(const StepBuffers& b, const double* lsrc, void* out, int64_t N, double u0,
                                   int mode, int keep, cudaStream_t s) {
  const unsigned ntiles = (unsigned)((N + SCAN_TILE - 1) / SCAN_TILE);
  const int sq = weight_scale_bits(N);
  T* o = static_cast<T*>(out);
  switch (mode) {
    case WSRC_BINS:
      k_scan_resample<T, WSRC_BINS><<<ntiles, SCAN_THREADS, 0, s>>>(b, lsrc, o, N, u0, sq, keep);
      break;
    default:
      k_scan_resample<T, WSRC_PARTICLES><<<ntiles, SCAN_THREADS, 0, s>>>(b, lsrc ? lsrc : b.ll, o, N, u0, sq,
                                                                         keep);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_resample(const StepBuffers& b, int dtype, void* state_out, int64_t N, double u0, int mode,
                            int keep, int num_sms, cudaStream_t s) {
  (void)num_sms;
  return dtype == PCSIR_F32 ? resample_launch<float>(b, nullptr, state_out, N, u0, mode, keep, s)
                            : resample_launch<double>(b, nullptr, state_out, N, u0, mode, keep, s);
}

cudaError_t launch_resample_logw(const StepBuffers& b, const double* logw, int32_t* anc_out, int64_t N, double u0,
                                 cudaStream_t s) {
  // ancestors only, no state gather
  StepBuffers bb = b;
  bb.anc = anc_out;
  return resample_launch<float>(bb, logw, nullptr, N, u0, WSRC_PARTICLES, PCSIR_KEEP_ANCESTORS, s);
}

}  // namespace pcsir
