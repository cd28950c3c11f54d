// Systematic resampling (Algorithm 1/2 resampling step): integer weights, a
// tile-level prefix scan, and the gather of the selected propagated states
// into the caller's buffer.
//
// Weights enter as integers q_i = rint(exp(ll_i - max) 2^sq), so the
// cumulative sums C_j are exact and independent of the summation order.
// Output i takes the first particle j with C_j > U_i, where
// U_i = (i + u0) T / N and T = C_{N-1}; U_i is evaluated in 64.64 fixed point
// as i * Delta + U0 with Delta = T / N and U0 = u0 * Delta, and only its
// integer part is compared with the integer C_j, which decides C_j > U_i
// exactly.  Each tile of particles owns the outputs whose U falls between its
// exclusive and inclusive prefixes, so every output is written exactly once.
//
// Two kernels: k_tile_sums (k_tile_sums_bins, on a resident grid, for pcSIR
// steps) adds up each tile's integer weights and its last block scans the
// tile sums, fixes the 64.64 map and each tile's output range; k_resample
// then scans within each tile and gives every output its ancestor by binary
// search over the tile's cumulative weights.  A tile whose particles carry a
// large share of the weight (all of it, when one particle dominates) owns
// many outputs: they are split into chunks of RS_CHUNK over extra blocks, so
// the time of the step does not depend on how the weight is spread.  No block
// ever waits for another.
#include <cmath>
#include <type_traits>

#include "pcsir_device.cuh"

namespace pcsir {

struct Map64 {
  unsigned long long dhi, dlo, uhi, ulo;
};

// integer part of i * Delta + U0
__device__ __forceinline__ long long u_int(const Map64& mp, long long i) {
  const unsigned long long ui = (unsigned long long)i;
  const unsigned long long plo = ui * mp.dlo;
  const unsigned long long phi = __umul64hi(ui, mp.dlo);
  const unsigned long long s = plo + mp.ulo;
  const unsigned long long carry = s < plo ? 1ull : 0ull;
  return (long long)(ui * mp.dhi + mp.uhi + phi + carry);
}

// first output index i in [0, N] with U_i >= C (N if none): a float guess of
// (C - U0) / Delta, then the exact integer correction
__device__ long long first_out_f(const Map64& mp, long long C, long long N, float inv_delta) {
  if (C <= 0) return 0;
  if (mp.dhi == 0ull && mp.dlo == 0ull) return N;
  long long back;
  const float cf = i64_trunc_float(C - (long long)mp.uhi, &back);
  float xf = __fmul_rn(cf, inv_delta);
  long long i = xf <= 0.0f ? 0 : (xf >= (float)N ? N : (long long)__float2int_rn(xf));
  int guard = 0;
  while (i > 0 && u_int(mp, i - 1) >= C && guard++ < 256) --i;
  while (i < N && u_int(mp, i) < C && guard++ < 512) ++i;
  return i;
}

// i * Delta + U0 in full (integer part hi, fraction lo), and the sum of two such values
struct U128 {
  unsigned long long hi, lo;
};
__device__ __forceinline__ U128 u_full(const Map64& mp, unsigned long long i) {
  const unsigned long long plo = i * mp.dlo;
  const unsigned long long lo = plo + mp.ulo;
  return U128{i * mp.dhi + mp.uhi + __umul64hi(i, mp.dlo) + (lo < plo ? 1ull : 0ull), lo};
}
__device__ __forceinline__ U128 u_add(U128 a, U128 b) {
  const unsigned long long lo = a.lo + b.lo;
  return U128{a.hi + b.hi + (lo < a.lo ? 1ull : 0ull), lo};
}

// two consecutive values at an 8-byte (float) or 16-byte (double) aligned address
__device__ __forceinline__ void store_pair(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void store_pair(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

__device__ __forceinline__ Map64 load_map(const Control* ctl) {
  Map64 mp;
  mp.dhi = ctl->delta_hi;
  mp.dlo = ctl->delta_lo;
  mp.uhi = ctl->u0_hi;
  mp.ulo = ctl->u0_lo;
  return mp;
}

__device__ __forceinline__ int pad_idx(int j) { return j + (j >> 4); }

// A resampling block writes at most RS_CHUNK outputs: a tile that owns more (its particles carry
// more than RS_CHUNK / N of the total weight, up to all of it) has its further outputs written
// by extra blocks, one per chunk, so that no block serialises a large share of the N outputs.
// The extra blocks launched, ceil(N / RS_CHUNK), cover every case: the further chunks of all
// tiles number at most N / RS_CHUNK.
constexpr long long RS_CHUNK = 4LL * SCAN_TILE;

__device__ __forceinline__ int rs_extra_chunks(long long n) { return n > RS_CHUNK ? (int)((n - 1) / RS_CHUNK) : 0; }

// Number of the tile's cumulative weights C_j <= u (j < SCAN_TILE), by a fixed
// 12-step binary search over Cs in the padded layout (index j at j + j / 16).
// While the search adds steps >= 16 the position a stays a multiple of 16, so
// the probe a + step - 1 sits at pa + (step - 1) + (step - 1) / 16 with
// pa = a + a / 16; the smaller steps never cross a pad.  Every probe is thus
// the running padded position plus a constant.
__device__ __forceinline__ int tile_search(const long long* __restrict__ Cs, long long u) {
  int pa = 0;
#pragma unroll
  for (int step = SCAN_TILE / 2; step > 0; step >>= 1)
    if (Cs[pa + (step - 1) + ((step - 1) >> 4)] <= u) pa += step + (step >> 4);
  return pa - pa / 17;  // pa = 17 (a / 16) + a % 16
}

// every map entry is written before it is read; the clamp only keeps a
// gather inside the tile should that ever fail
__device__ __forceinline__ int clamp_item(int a, int cnt) { return a < 0 ? 0 : (a >= cnt ? cnt - 1 : a); }

// Integer weights of the tile's particles j = 1024 k + 4 t + e: WSRC_BINS reads
// the particle's hash slot and the bin's q; otherwise q is computed from the
// particle's log-weight.  Particles past the end weigh 0.
template <int WSRC>
__device__ __forceinline__ long long src_llq(const StepBuffers& b, const double* __restrict__ lsrc, int64_t i) {
  return WSRC == WSRC_LOGW ? llq_of(lsrc[i]) : b.llq[i];  // WSRC_PARTICLES, WSRC_Q
}

template <int WSRC>
__device__ __forceinline__ void tile_weights(const StepBuffers& b, const double* __restrict__ lsrc, int64_t base,
                                             int cnt, long long mq, bool any, int sq, long long q[SCAN_ITEMS]) {
  const int tid = threadIdx.x;
  if (WSRC == WSRC_BINS) {
    unsigned g[SCAN_ITEMS];
    const bool vec = cnt == SCAN_TILE;
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
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) q[k] = g[k] != 0xffffffffu ? b.hq[g[k]] : 0ll;
  } else if (WSRC == WSRC_Q) {
    // 16-byte loads of four consecutive integer weights (tile starts are 32-byte aligned)
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS / 4; ++k) {
      const int j0 = k * (4 * SCAN_THREADS) + 4 * tid;
      if (j0 + 4 <= cnt) {
        const longlong2 a = *reinterpret_cast<const longlong2*>(b.hq + base + j0);
        const longlong2 c = *reinterpret_cast<const longlong2*>(b.hq + base + j0 + 2);
        q[4 * k] = a.x;
        q[4 * k + 1] = a.y;
        q[4 * k + 2] = c.x;
        q[4 * k + 3] = c.y;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) q[4 * k + e] = (j0 + e < cnt) ? b.hq[base + j0 + e] : 0ll;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS / 4; ++k) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = k * (4 * SCAN_THREADS) + 4 * tid + e;
        q[4 * k + e] = (j < cnt && any) ? q_of_wtilde(wtilde_q(src_llq<WSRC>(b, lsrc, base + j), mq), sq) : 0ll;
      }
    }
  }
}

__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Per-tile sums of the integer weights; the last block scans them into the
// tiles' exclusive prefixes and fixes Delta and U0.
// ---------------------------------------------------------------------------
// The last block to finish its tiles: exclusive scan of the nt tile sums into the tiles'
// prefixes, then Delta = T / N, U0 = u0 Delta (64.64 fixed point) and the FP32 reciprocal, and
// the tiles' output ranges: tile t owns the outputs i with excl_t <= U_i < excl_{t+1}, i.e.
// [tile_lo[t], tile_lo[t + 1]), and the outputs past its first RS_CHUNK form further chunks,
// whose exclusive prefix over the tiles goes to tile_ovx.
__device__ void tile_scan_tail(const StepBuffers& b, Control* ctl, int64_t N, double u0, int nt,
                               long long* wtot) {
  __shared__ Map64 s_mp;
  __shared__ float s_inv;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // exclusive scan of the tile sums (each thread a run of consecutive tiles)
  const int per = (nt + SCAN_THREADS - 1) / SCAN_THREADS;
  const int t0 = tid * per;
  long long run = 0;
  for (int k = 0; k < per && t0 + k < nt; ++k) run += *(volatile long long*)&b.tile_sum[t0 + k];
  long long inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wtot[w] = inc;
  __syncthreads();
  long long off = 0, total = 0;
  for (int j = 0; j < SCAN_THREADS / 32; ++j) {
    if (j < w) off += wtot[j];
    total += wtot[j];
  }
  long long e = off + inc - run;
  for (int k = 0; k < per && t0 + k < nt; ++k) {
    const long long v = *(volatile long long*)&b.tile_sum[t0 + k];
    b.tile_excl[t0 + k] = e;
    e += v;
  }
  if (tid == 0) {
    // Delta = T / N and U0 = u0 Delta in 64.64 fixed point
    const unsigned long long T = (unsigned long long)total;
    const unsigned long long n = (unsigned long long)N;
    const unsigned long long dhi = T / n;
    const unsigned long long rem = T % n;
    const unsigned long long dlo = (unsigned long long)(((unsigned __int128)rem << 64) / n);
    double uf = u0 * 18446744073709551616.0;
    if (!(uf >= 0.0)) uf = 0.0;
    const unsigned long long u0f = uf >= 18446744073709549568.0 ? 18446744073709549568ull : __double2ull_rz(uf);
    const unsigned __int128 tot = (unsigned __int128)u0f * dhi + (((unsigned __int128)u0f * dlo) >> 64);
    ctl->delta_hi = dhi;
    ctl->delta_lo = dlo;
    ctl->u0_hi = (unsigned long long)(tot >> 64);
    ctl->u0_lo = (unsigned long long)tot;
    const double dd = (double)dhi + (double)dlo * 5.421010862427522e-20;
    ctl->inv_delta = dd > 0.0 ? (float)(1.0 / dd) : 0.0f;
    s_mp.dhi = dhi;
    s_mp.dlo = dlo;
    s_mp.uhi = (unsigned long long)(tot >> 64);
    s_mp.ulo = (unsigned long long)tot;
    s_inv = ctl->inv_delta;
    if (T == 0ull) atomicOr(&ctl->err, (unsigned)PCSIR_DERR_ZEROSUM);
  }
  __syncthreads();
  // A tile with tile_sum N < (RS_CHUNK - 2) T owns fewer than RS_CHUNK outputs (U_i advances by
  // T / N per output).  When every tile is such, the output ranges are left to the resampling
  // blocks themselves (tile_ovx[nt] = -1: no further chunks); otherwise they are fixed here.
  bool big = false;
  for (int k = 0; k < per && t0 + k < nt; ++k) {
    const unsigned long long v = (unsigned long long)*(volatile long long*)&b.tile_sum[t0 + k];
    big |= (unsigned __int128)v * (unsigned long long)N >=
           (unsigned __int128)(unsigned long long)(RS_CHUNK - 2) * (unsigned long long)total;
  }
  if (!__syncthreads_or(big)) {
    if (tid == 0) b.tile_ovx[nt] = -1;
    return;
  }
  // first output of each tile (the last entry: N)
  const Map64 mp = s_mp;
  const float inv = s_inv;
  for (int k = 0; k < per && t0 + k < nt; ++k) b.tile_lo[t0 + k] = first_out_f(mp, b.tile_excl[t0 + k], N, inv);
  if (tid == 0) b.tile_lo[nt] = N;
  __syncthreads();  // also orders this block's global writes above before the reads below
  // chunks past the first of each tile, and their exclusive prefix
  int cnt = 0;
  for (int k = 0; k < per && t0 + k < nt; ++k) cnt += rs_extra_chunks(b.tile_lo[t0 + k + 1] - b.tile_lo[t0 + k]);
  int ci = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, ci, o);
    if (lane >= o) ci += v;
  }
  if (lane == 31) wtot[w] = ci;  // every thread read wtot before the barriers above
  __syncthreads();
  int coff = 0, ctot = 0;
  for (int j = 0; j < SCAN_THREADS / 32; ++j) {
    if (j < w) coff += (int)wtot[j];
    ctot += (int)wtot[j];
  }
  int ce = coff + ci - cnt;
  for (int k = 0; k < per && t0 + k < nt; ++k) {
    b.tile_ovx[t0 + k] = ce;
    ce += rs_extra_chunks(b.tile_lo[t0 + k + 1] - b.tile_lo[t0 + k]);
  }
  if (tid == 0) b.tile_ovx[nt] = ctot;
}

template <int WSRC>
__global__ void __launch_bounds__(SCAN_THREADS)
k_tile_sums(StepBuffers b, const double* __restrict__ lsrc, int64_t N, double u0, int sq) {
  __shared__ long long red[SCAN_THREADS / 32];
  __shared__ long long wtot[SCAN_THREADS / 32];
  __shared__ bool last;
  Control* ctl = b.ctl;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const int cnt = (int)((N - base) < SCAN_TILE ? (N - base) : SCAN_TILE);
  const unsigned long long me = ctl->max_llq;
  long long q[SCAN_ITEMS];
  tile_weights<WSRC>(b, lsrc, base, cnt, llq_dec(me), me != 0ull, sq, q);
  long long t = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) t += q[k];
  t = warp_sum_i64(t);
  if (lane == 0) red[w] = t;
  __syncthreads();
  if (tid == 0) {
    long long s = 0;
    for (int j = 0; j < SCAN_THREADS / 32; ++j) s += red[j];
    b.tile_sum[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(&ctl->tsum_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  tile_scan_tail(b, ctl, N, u0, (int)gridDim.x, wtot);
}

// pcSIR tile sums with a resident grid: each block runs over tiles blockIdx.x, + gridDim.x, ...,
// the slots of its next tile loaded before the current tile's cell weights are gathered, so that
// the slot reads stay in flight while blocks reduce
__device__ __forceinline__ void load_tile_slots(const StepBuffers& b, int64_t N, int tile, uint4 g[SCAN_ITEMS / 4]) {
  const int64_t base = (int64_t)tile * SCAN_TILE;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS / 4; ++k) {
    const int64_t j = base + k * (4 * SCAN_THREADS) + 4 * threadIdx.x;
    if (j + 4 <= N) {
      g[k] = *reinterpret_cast<const uint4*>(b.pslot + j);
    } else {
      g[k].x = j < N ? b.pslot[j] : 0xffffffffu;
      g[k].y = j + 1 < N ? b.pslot[j + 1] : 0xffffffffu;
      g[k].z = j + 2 < N ? b.pslot[j + 2] : 0xffffffffu;
      g[k].w = j + 3 < N ? b.pslot[j + 3] : 0xffffffffu;
    }
  }
}

constexpr int TS_BLOCKS_PER_SM = 6;  // resident tile-sum blocks per SM (40 registers, 256 threads)

__global__ void __launch_bounds__(SCAN_THREADS, TS_BLOCKS_PER_SM) k_tile_sums_bins(StepBuffers b, int64_t N, double u0, int ntiles) {
  __shared__ long long red[2][SCAN_THREADS / 32];
  __shared__ long long wtot[SCAN_THREADS / 32];
  __shared__ bool last;
  Control* ctl = b.ctl;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  uint4 cur[SCAN_ITEMS / 4], nxt[SCAN_ITEMS / 4];
  if ((int)blockIdx.x < ntiles) load_tile_slots(b, N, blockIdx.x, cur);
  int parity = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, parity ^= 1) {
    const int next = tile + (int)gridDim.x;
    if (next < ntiles) load_tile_slots(b, N, next, nxt);
    long long t = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS / 4; ++k) {
      const unsigned gs[4] = {cur[k].x, cur[k].y, cur[k].z, cur[k].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) t += gs[e] != 0xffffffffu ? b.hq[gs[e]] : 0ll;
    }
    t = warp_sum_i64(t);
    // two halves of the partials alternate, so one barrier per tile separates writes and reads
    if (lane == 0) red[parity][w] = t;
    __syncthreads();
    if (tid == 0) {
      long long s = 0;
      for (int j = 0; j < SCAN_THREADS / 32; ++j) s += red[parity][j];
      b.tile_sum[tile] = s;
    }
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS / 4; ++k) cur[k] = nxt[k];
  }
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(&ctl->tsum_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  tile_scan_tail(b, ctl, N, u0, ntiles, wtot);
}

// ---------------------------------------------------------------------------
// Resampling of one tile: inclusive cumulative weights of the tile in shared
// memory, then the tile's outputs i (those with C_{-1} <= U_i < C_{cnt-1}),
// each finding by binary search the particle k with C_{k-1} <= U_i < C_k and
// gathering its propagated state.  Blocks [0, ntiles) take tile blockIdx.x and
// its first RS_CHUNK outputs; the blocks past them take the further chunks of
// the tiles that own more outputs, in tile order (tile_ovx), and exit when
// there are fewer such chunks than blocks.
// ---------------------------------------------------------------------------
template <typename T, int WSRC, int NS = 5>
__global__ void __launch_bounds__(SCAN_THREADS, 5)
k_resample(StepBuffers b, const double* __restrict__ lsrc, T* __restrict__ out, int64_t N, int sq, int keep,
           int ntiles) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  long long* Cs = reinterpret_cast<long long*>(rs_smem);                       // SCAN_TILE + SCAN_TILE / 16
  __shared__ long long wtot[SCAN_THREADS / 32];
  __shared__ long long s_lo, s_hi;
  __shared__ int s_tile;
  Control* ctl = b.ctl;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    // this block's tile and outputs [s_lo, s_hi): the first RS_CHUNK outputs of tile blockIdx.x, or
    // extra chunk e = blockIdx.x - ntiles: chunk e - tile_ovx[t] + 1 of the tile t with
    // tile_ovx[t] <= e < tile_ovx[t + 1] (the largest such t); none when e is past them all
    int t = (int)blockIdx.x;
    long long chunk = 0;
    bool idle = false;
    if (t >= ntiles) {
      const int e = t - ntiles;
      idle = e >= b.tile_ovx[ntiles];
      int lo = 0, hi = ntiles - 1;
      while (!idle && lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.tile_ovx[mid] <= e) lo = mid;
        else hi = mid - 1;
      }
      t = idle ? 0 : lo;
      chunk = idle ? 0 : (long long)(e - b.tile_ovx[lo]) + 1;
    }
    long long t_lo, t_hi;
    if (b.tile_ovx[ntiles] < 0) {
      // every tile owns fewer than RS_CHUNK outputs: its range from the first-output search
      const Map64 m = load_map(ctl);
      t_lo = first_out_f(m, b.tile_excl[t], N, ctl->inv_delta);
      t_hi = t == ntiles - 1 ? N : first_out_f(m, b.tile_excl[t + 1], N, ctl->inv_delta);
    } else {
      t_lo = b.tile_lo[t];
      t_hi = b.tile_lo[t + 1];
    }
    const long long lo = t_lo + chunk * RS_CHUNK;
    s_tile = idle ? -1 : t;
    s_lo = lo;
    s_hi = idle ? lo : (t_hi < lo + RS_CHUNK ? t_hi : lo + RS_CHUNK);
  }
  __syncthreads();
  const bool idle = s_tile < 0;
  const bool primary = (int)blockIdx.x < ntiles;
  const int tile = idle ? 0 : s_tile;
  const int64_t base = (int64_t)tile * SCAN_TILE;
  const int cnt = (int)((N - base) < SCAN_TILE ? (N - base) : SCAN_TILE);
  const unsigned long long me = ctl->max_llq;
  const long long mq = llq_dec(me);
  const size_t hcap = size_t(1) << b.hbits;
  const Map64 mp = load_map(ctl);
  const long long excl = b.tile_excl[tile];

  // ESS-thresholded steps (lw_out set): the particles are resampled only when N_eff < ess_min,
  // from the weight sums of this step (the same for every block)
  bool skip = false;
  if (b.lw_out != nullptr) {
    const double Tf = *(volatile double*)&ctl->T_f, T2 = *(volatile double*)&ctl->T2_f;
    skip = !(Tf * Tf / T2 < b.ess_min);
  }
  if (idle) {
    // no outputs left for this block
  } else if (skip) {
    // no resampling: the propagated particles and their log-weights (minus the maximum)
    // carry over to the next step (the tile's own block only)
    const T* __restrict__ prop = static_cast<const T*>(b.prop);
    for (int j = tid; primary && j < cnt; j += SCAN_THREADS) {
      const int64_t i = base + j;
      if (out != nullptr) {
#pragma unroll
        for (int d = 0; d < NS; ++d) out[d * N + i] = prop[d * N + i];
      }
      const long long q = b.llq[i];
      b.lw_out[i] = q == LLQ_NONE ? LLQ_NONE : q - mq;
      if (keep & PCSIR_KEEP_ANCESTORS) b.anc[i] = (int32_t)i;
    }
  } else {
    // 1. integer weights, into padded shared memory in particle order
    {
      long long q[SCAN_ITEMS];
      tile_weights<WSRC>(b, lsrc, base, cnt, mq, me != 0ull, sq, q);
#pragma unroll
      for (int k = 0; k < SCAN_ITEMS / 4; ++k) {
        const int j0 = k * (4 * SCAN_THREADS) + 4 * tid;
#pragma unroll
        for (int e = 0; e < 4; ++e) Cs[pad_idx(j0 + e)] = q[4 * k + e];
      }
    }
    __syncthreads();
    // 2. each thread's total of its ITEMS consecutive weights (the running sums are formed again in
    //    step 4 from shared memory rather than held in 2 x ITEMS registers, for residency)
    long long run = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) run += Cs[pad_idx(tid * SCAN_ITEMS + k)];
    // 3. exclusive scan of the thread totals across the block
    long long inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane == 31) wtot[w] = inc;
    __syncthreads();
    long long woff = 0;
#pragma unroll
    for (int j = 0; j < SCAN_THREADS / 32; ++j)
      if (j < w) woff += wtot[j];
    const long long texcl = woff + inc - run;
    // 4. inclusive cumulative weights C_j of the tile; entries past its last particle compare
    //    above every U_i (the fixed-step search below)
    {
      long long c = excl + texcl;
#pragma unroll
      for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int jj = tid * SCAN_ITEMS + k;
        c += Cs[pad_idx(jj)];  // this thread's own items: no other thread reads or writes them here
        Cs[pad_idx(jj)] = jj < cnt ? c : LLONG_MAX;
      }
    }
    __syncthreads();
    // 5. the tile's outputs, two per thread and pass.  Output i's ancestor is the particle j with
    //    C_{j-1} <= U_i < C_j, i.e. the number of C_j <= floor(U_i) (the C_j are integers): a
    //    12-step search over the tile's cumulative weights in shared memory, or for the second
    //    output of a pair at most WALK comparisons before it; every output costs a bounded number
    //    of steps, so a particle with many offspring does not serialise one thread.  Row offsets
    //    fit 32 bits (N <= 2^26).
    // the tile's outputs are [tile_lo[t], tile_lo[t + 1]) (U >= C_{-1} = excl and U < C_{cnt-1}, the
    // next tile's excl); this block writes its chunk [s_lo, s_hi) of them
    const T* __restrict__ prop = static_cast<const T*>(b.prop);
    const long long lo = s_lo, hi = s_hi;
    const bool zero_sum = (mp.dhi == 0ull && mp.dlo == 0ull);
    const unsigned nb = (unsigned)N;
    const unsigned ub = (unsigned)base;
    if (out == nullptr) {
      // ancestors only (deferred resampling, the stand-alone calls): two outputs SCAN_THREADS
      // apart per thread and pass, each by the fixed-step search (measured faster here than the
      // pairs below, whose walk pays only where the states are gathered too)
      constexpr int RO = 2;
      // U of the thread's outputs r0 and r0 + SCAN_THREADS, advanced by RO SCAN_THREADS Delta per pass
      // (exact 128-bit additions instead of a product per output)
      const U128 d1 = u_full(Map64{mp.dhi, mp.dlo, 0ull, 0ull}, (unsigned long long)SCAN_THREADS);
      const U128 d2 = u_add(d1, d1);
      U128 u0r = u_full(mp, (unsigned long long)(lo + tid));
      for (long long r0 = lo + tid; r0 < hi; r0 += RO * SCAN_THREADS, u0r = u_add(u0r, d2)) {
        unsigned ii[RO], aa[RO];
        bool has[RO];
#pragma unroll
        for (int j = 0; j < RO; ++j) {
          const long long i = r0 + (long long)j * SCAN_THREADS;
          has[j] = i < hi;
          ii[j] = (unsigned)i;
          int a = 0;
          if (has[j] && !zero_sum) a = tile_search(Cs, (long long)(j == 0 ? u0r : u_add(u0r, d1)).hi);
          // all weights zero (Delta = 0): no distribution to sample, keep every particle
          aa[j] = has[j] ? (zero_sum ? ii[j] : ub + (unsigned)clamp_item(a, cnt)) : 0u;
        }
        if (keep & PCSIR_KEEP_ANCESTORS) {
#pragma unroll
          for (int j = 0; j < RO; ++j)
            if (has[j]) b.anc[ii[j]] = (int32_t)aa[j];
        }
        // resampled particles restart from uniform weights
        if (b.lw_out != nullptr) {
#pragma unroll
          for (int j = 0; j < RO; ++j)
            if (has[j]) b.lw_out[ii[j]] = 0;
        }
      }
    } else {
      // each thread takes two consecutive outputs r0, r0 + 1 per pass (r0 even): the first ancestor
      // by the search, the second by walking on from it over the few cumulative weights up to
      // U_{r0+1} = U_{r0} + Delta (a search again after WALK steps), so that most outputs cost a
      // comparison or two instead of twelve.  The two outputs' states leave with one 8-byte store per
      // component where the rows allow it.
      constexpr int WALK = 4;
      const long long lo2 = lo & ~1ll;
      const bool pair_st = (N & 1) == 0 && (reinterpret_cast<uintptr_t>(out) & (2 * sizeof(T) - 1)) == 0;
      // a caller's ancestor array may start off an 8-byte boundary
      const bool pair_anc = (reinterpret_cast<uintptr_t>(b.anc) & 7) == 0;
      const U128 dd = u_full(Map64{mp.dhi, mp.dlo, 0ull, 0ull}, 1ull);
      const U128 dstep = u_full(Map64{mp.dhi, mp.dlo, 0ull, 0ull}, 2ull * SCAN_THREADS);
      U128 ur = u_full(mp, (unsigned long long)(lo2 + 2 * tid));
      for (long long r0 = lo2 + 2 * tid; r0 < hi; r0 += 2 * SCAN_THREADS, ur = u_add(ur, dstep)) {
        const bool h0 = r0 >= lo, h1 = r0 + 1 < hi;
        int a0 = 0, a1 = 0;
        if (!zero_sum) {
          a0 = tile_search(Cs, (long long)ur.hi);
          const long long u1 = (long long)u_add(ur, dd).hi;
          a1 = a0;
          int k = 0;
          while (k < WALK && Cs[pad_idx(a1)] <= u1) {  // entries past the tile's end are LLONG_MAX
            ++a1;
            ++k;
          }
          if (k == WALK && Cs[pad_idx(a1)] <= u1) a1 = tile_search(Cs, u1);
        }
        const unsigned i0 = (unsigned)r0;
        // all weights zero (Delta = 0): no distribution to sample, keep every particle
        const unsigned s0 = zero_sum ? i0 : ub + (unsigned)clamp_item(a0, cnt);
        const unsigned s1 = zero_sum ? i0 + 1u : ub + (unsigned)clamp_item(a1, cnt);
        T v0[NS], v1[NS];
#pragma unroll
        for (int d = 0; d < NS; ++d) {
          v0[d] = h0 ? prop[d * nb + s0] : T(0);
          v1[d] = h1 ? prop[d * nb + s1] : T(0);
        }
        if (pair_st && h0 && h1) {
#pragma unroll
          for (int d = 0; d < NS; ++d) store_pair(out + d * nb + i0, v0[d], v1[d]);
        } else {
#pragma unroll
          for (int d = 0; d < NS; ++d) {
            if (h0) out[d * nb + i0] = v0[d];
            if (h1) out[d * nb + i0 + 1u] = v1[d];
          }
        }
        if (keep & PCSIR_KEEP_ANCESTORS) {
          if (h0 && h1 && pair_anc) {
            *reinterpret_cast<int2*>(b.anc + i0) = make_int2((int)s0, (int)s1);  // i0 even
          } else {
            if (h0) b.anc[i0] = (int32_t)s0;
            if (h1) b.anc[i0 + 1u] = (int32_t)s1;
          }
        }
        // resampled particles restart from uniform weights
        if (b.lw_out != nullptr) {
          if (h0) b.lw_out[i0] = 0;
          if (h1) b.lw_out[i0 + 1u] = 0;
        }
      }
    }
  }
  // 6. optional per-particle outputs of the tile (its own block)
  if (primary && (keep & (PCSIR_KEEP_WEIGHTS | PCSIR_KEEP_PARTICLE_BIN | PCSIR_KEEP_QWEIGHTS))) {
    const double Tf = *(volatile double*)&ctl->T_f;
    for (int j = tid; j < cnt; j += SCAN_THREADS) {
      const int64_t i = base + j;
      if (WSRC == WSRC_BINS) {
        const unsigned g = b.pslot[i];
        if (keep & PCSIR_KEEP_WEIGHTS) b.wout[i] = b.hw[g] / Tf;
        if (keep & PCSIR_KEEP_PARTICLE_BIN) b.pbin[i] = b.hrank[g];
        if (keep & PCSIR_KEEP_QWEIGHTS) b.qout[i] = b.hq[g];
      } else {
        const df wd = me == 0ull ? df{0.0f, 0.0f} : wtilde_q(src_llq<WSRC>(b, lsrc, i), mq);
        if (keep & PCSIR_KEEP_WEIGHTS) b.wout[i] = ((double)wd.hi + (double)wd.lo) / Tf;
        if (keep & PCSIR_KEEP_QWEIGHTS)
          b.qout[i] = WSRC == WSRC_Q ? b.hq[i] : (me == 0ull ? 0ll : q_of_wtilde(wd, sq));
      }
    }
  }
  // 7. pcSIR: return the occupied hash slots to empty for the next step
  if (WSRC == WSRC_BINS && primary) {
    const unsigned B = ctl->nocc;
    for (unsigned bi = tile * SCAN_THREADS + tid; bi < B; bi += (unsigned)ntiles * SCAN_THREADS) {
      const unsigned g = b.occ[bi];
      b.hkey[g] = EMPTY_KEY;
      b.hcnt[g] = 0u;
#pragma unroll
      for (int d = 0; d < NS; ++d) b.hsum[d * hcap + g] = 0;
    }
  }
  // 8. the last tile to finish publishes the step's device error flags
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&ctl->tiles_done, 1u) == gridDim.x - 1) {
      __threadfence();
      *b.derr_out = (int32_t)(*(volatile unsigned*)&ctl->err);
      if (b.resampled_out != nullptr) *b.resampled_out = skip ? 0 : 1;
    }
  }
}

constexpr size_t RS_SMEM = sizeof(long long) * (SCAN_TILE + SCAN_TILE / 16);

// resampling grid: one block per tile, then ceil(N / RS_CHUNK) blocks for further output chunks
static unsigned rs_grid(int64_t N) {
  return (unsigned)((N + SCAN_TILE - 1) / SCAN_TILE + (N + RS_CHUNK - 1) / RS_CHUNK);
}

cudaError_t prepare_resample() {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_resample<float, WSRC_BINS>, a, (int)RS_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resample<float, WSRC_PARTICLES>, a, (int)RS_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resample<float, WSRC_LOGW>, a, (int)RS_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resample<double, WSRC_BINS>, a, (int)RS_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resample<double, WSRC_PARTICLES>, a, (int)RS_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resample<double, WSRC_LOGW>, a, (int)RS_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resample<float, WSRC_Q>, a, (int)RS_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resample<float, WSRC_BINS, 7>, a, (int)RS_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resample<float, WSRC_PARTICLES, 7>, a, (int)RS_SMEM);
  return e;
}

template <typename T>
static cudaError_t resample_launch(const StepBuffers& b, const double* lsrc, void* out, int64_t N, double u0,
                                   int mode, int keep, cudaStream_t s, int num_sms = 0) {
  const unsigned ntiles = (unsigned)((N + SCAN_TILE - 1) / SCAN_TILE);
  const int sq = weight_scale_bits(N);
  T* o = static_cast<T*>(out);
  if (mode == WSRC_BINS) {
    if (num_sms > 0) {
      const unsigned grid = ntiles < (unsigned)(num_sms * TS_BLOCKS_PER_SM) ? ntiles : (unsigned)(num_sms * TS_BLOCKS_PER_SM);
      k_tile_sums_bins<<<grid, SCAN_THREADS, 0, s>>>(b, N, u0, (int)ntiles);
    } else {
      k_tile_sums<WSRC_BINS><<<ntiles, SCAN_THREADS, 0, s>>>(b, lsrc, N, u0, sq);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_resample<T, WSRC_BINS><<<rs_grid(N), SCAN_THREADS, RS_SMEM, s>>>(b, lsrc, o, N, sq, keep, (int)ntiles);
  } else if (mode == WSRC_PARTICLES) {
    k_tile_sums<WSRC_PARTICLES><<<ntiles, SCAN_THREADS, 0, s>>>(b, nullptr, N, u0, sq);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_resample<T, WSRC_PARTICLES><<<rs_grid(N), SCAN_THREADS, RS_SMEM, s>>>(b, nullptr, o, N, sq, keep, (int)ntiles);
  } else if (mode == WSRC_Q) {
    if (!std::is_same<T, float>::value) return cudaErrorInvalidValue;  // FP32 state only
    k_tile_sums<WSRC_Q><<<ntiles, SCAN_THREADS, 0, s>>>(b, nullptr, N, u0, sq);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_resample<float, WSRC_Q><<<rs_grid(N), SCAN_THREADS, RS_SMEM, s>>>(b, nullptr, reinterpret_cast<float*>(o), N,
                                                                       sq, keep, (int)ntiles);
  } else {
    k_tile_sums<WSRC_LOGW><<<ntiles, SCAN_THREADS, 0, s>>>(b, lsrc, N, u0, sq);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_resample<T, WSRC_LOGW><<<rs_grid(N), SCAN_THREADS, RS_SMEM, s>>>(b, lsrc, o, N, sq, keep, (int)ntiles);
  }
  return cudaGetLastError();
}

cudaError_t launch_resample(const StepBuffers& b, int dtype, void* state_out, int64_t N, double u0, int mode,
                            int keep, int num_sms, cudaStream_t s) {
  return dtype == PCSIR_F32 ? resample_launch<float>(b, nullptr, state_out, N, u0, mode, keep, s, num_sms)
                            : resample_launch<double>(b, nullptr, state_out, N, u0, mode, keep, s, num_sms);
}

cudaError_t launch_resample7(const StepBuffers& b, float* state_out, int64_t N, double u0, int mode, int keep,
                             cudaStream_t s) {
  const unsigned ntiles = (unsigned)((N + SCAN_TILE - 1) / SCAN_TILE);
  const int sq = weight_scale_bits(N);
  if (mode == WSRC_BINS) {
    k_tile_sums<WSRC_BINS><<<ntiles, SCAN_THREADS, 0, s>>>(b, nullptr, N, u0, sq);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_resample<float, WSRC_BINS, 7><<<rs_grid(N), SCAN_THREADS, RS_SMEM, s>>>(b, nullptr, state_out, N, sq, keep,
                                                                             (int)ntiles);
  } else {
    k_tile_sums<WSRC_PARTICLES><<<ntiles, SCAN_THREADS, 0, s>>>(b, nullptr, N, u0, sq);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_resample<float, WSRC_PARTICLES, 7><<<rs_grid(N), SCAN_THREADS, RS_SMEM, s>>>(b, nullptr, state_out, N, sq,
                                                                                  keep, (int)ntiles);
  }
  return cudaGetLastError();
}

cudaError_t launch_resample_logw(const StepBuffers& b, const double* logw, int32_t* anc_out, int64_t N, double u0,
                                 cudaStream_t s) {
  // ancestors only, no state gather
  StepBuffers bb = b;
  bb.anc = anc_out;
  return resample_launch<float>(bb, logw, nullptr, N, u0, WSRC_LOGW, PCSIR_KEEP_ANCESTORS, s);
}

}  // namespace pcsir
