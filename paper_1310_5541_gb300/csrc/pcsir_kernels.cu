// Front half of a filter step: propagation, cells, dummies, likelihood and the
// weight reductions (Algorithm 1 / Algorithm 2 up to the resampling step).
#include <algorithm>
#include <type_traits>
#include <cfloat>
#include <cmath>

#include "pcsir_device.cuh"
#include "pcsir_philox.cuh"

namespace pcsir {

// ---------------------------------------------------------------------------
// State-precision arithmetic with explicit rounding (no contraction), so the
// propagated states and the cell indices are the IEEE results of the exact
// operation sequence x + vx + e and floor((x + 0.5) / h).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float floor_t(float a) { return floorf(a); }
__device__ __forceinline__ double floor_t(double a) { return floor(a); }
template <typename T> struct Scales;
template <> struct Scales<float> {
  static constexpr float POS = 2147483648.0f;  // 2^31
  static constexpr float VAL = 4194304.0f;     // 2^22
};
template <> struct Scales<double> {
  static constexpr double POS = 2147483648.0;
  static constexpr double VAL = 4194304.0;
};

// Nearly-constant-velocity transition of one particle (Section 5.1).
// With a resampling of the previous step left unapplied (src_idx), particle i
// of the resampled set is the propagated particle src_idx[i] of that step.
template <typename T>
__device__ __forceinline__ void propagate1(const T* __restrict__ st, const T* __restrict__ nz, int64_t N,
                                           int64_t i, T v[5], const int32_t* __restrict__ src_idx = nullptr) {
  const int64_t j = src_idx ? (int64_t)src_idx[i] : i;
  const T x = st[j], y = st[N + j], vx = st[2 * N + j], vy = st[3 * N + j], a = st[4 * N + j];
  const T ex = nz[i], ey = nz[N + i], evx = nz[2 * N + i], evy = nz[3 * N + i], ea = nz[4 * N + i];
  v[0] = add_rn(add_rn(x, vx), ex);
  v[1] = add_rn(add_rn(y, vy), ey);
  v[2] = add_rn(vx, evx);
  v[3] = add_rn(vy, evy);
  v[4] = add_rn(a, ea);
}

// The same with the increments drawn from the counter-based generator (FP32 state).
template <typename T>
__device__ __forceinline__ void propagate1_gen(const T* __restrict__ st, const NoiseGen& ng, int64_t N, int64_t i,
                                               T v[5], const int32_t* __restrict__ src_idx = nullptr) {
  const int64_t j = src_idx ? (int64_t)src_idx[i] : i;
  float e[5];
  ng_noise5(ng, i, e);
  const T x = st[j], y = st[N + j], vx = st[2 * N + j], vy = st[3 * N + j], a = st[4 * N + j];
  v[0] = add_rn(add_rn(x, vx), (T)e[0]);
  v[1] = add_rn(add_rn(y, vy), (T)e[1]);
  v[2] = add_rn(vx, (T)e[2]);
  v[3] = add_rn(vy, (T)e[3]);
  v[4] = add_rn(a, (T)e[4]);
}

__device__ __forceinline__ float abs_t(float a) { return fabsf(a); }
__device__ __forceinline__ double abs_t(double a) { return fabs(a); }

template <typename T>
__device__ __forceinline__ bool finite_state(const T v[5]) {
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 5; ++c) ok &= (abs_t(v[c]) < T(1.0e9));  // false for NaN / Inf too
  return ok;
}

// ---------------------------------------------------------------------------
// Global hash table over occupied cells.  Linear probing; a slot is claimed
// by CAS on its key and appended to the occupied list.  Capacity is at least
// twice the particle count, so the probe loop always terminates.
// ---------------------------------------------------------------------------
__device__ unsigned global_find_or_insert(const StepBuffers& b, unsigned long long key) {
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

// ---------------------------------------------------------------------------
// propagate + cell + centre-of-mass sums (pcSIR front, Algorithm 2).
//
// Each block keeps a private hash table of cells in shared memory.  For
// every cell it accumulates the member count and exact fixed-point sums of
// the five state components; the global table receives the block's partial
// sums with 64-bit integer atomics (exact and order-independent).
//   positions: offset from the cell origin in units of 2^-31 px (exact for
//              |x| >= 2^-8), biased by 2^33;
//   vx, vy, I0: offset from particle 0's input value in units of 2^-22,
//              biased by 2^34 (spread limit 2^12).
// A biased value is below 2^36 and is added as two 18-bit pieces to 32-bit
// shared-memory counters (64-bit shared atomics are an order of magnitude
// slower on this GPU); the counters are flushed to the global table at
// least every 2^14 particles, so no 32-bit counter can overflow.
// ---------------------------------------------------------------------------
constexpr int PB_THREADS = 512;
constexpr int PB_PER_THREAD = 4;
constexpr int PB_CHUNK = PB_THREADS * PB_PER_THREAD;
constexpr int PIECE_BITS = 18;
constexpr unsigned PIECE_MASK = (1u << PIECE_BITS) - 1u;
// A slot's 32-bit counters hold at most 2^14 particles' pieces (each < 2^18).
// A chunk adds at most CHUNK particles to one slot, so the table is flushed
// after any chunk that leaves some slot at 2^14 - CHUNK particles or more
// (the thread whose count crosses that mark raises the table's "hot" flag).
constexpr unsigned SLOT_PARTICLES = 1u << 14;
constexpr long long POS_BIAS = 1ll << 33;
constexpr long long VAL_BIAS = 1ll << 34;
constexpr long long BIASED_LIMIT = 1ll << 36;
constexpr int NACC = 11;  // count, then (lo, hi) of x, y, vx, vy, I0

// The block's table of cells: 2^LTB slots, filled to 3/4 at most.  Two sizes:
// 2^10 slots (56 KB, two blocks per SM) for cells that hold many particles,
// and 2^12 slots (224 KB, one block per SM) for small cells, where a block
// meets thousands of distinct cells and the small table would overflow into
// per-particle global atomics.
template <int LTB>
struct LocalTable {
  static constexpr int LT = 1 << LTB;
  static constexpr unsigned CAP = 3u << (LTB - 2);
  unsigned long long key[LT];
  unsigned int acc[NACC][LT];
  unsigned int gslot[LT];
  unsigned int fill;
  unsigned int hot;  // some slot may reach SLOT_PARTICLES within the next chunk: flush
};

// filled: set when this call's claim brought the table to its capacity (the table is emptied
// after the chunk)
template <int LTB>
__device__ __forceinline__ int local_find_or_insert(LocalTable<LTB>& t, unsigned long long key, bool& created,
                                                    bool& filled) {
  constexpr int LT = LocalTable<LTB>::LT;
  created = false;
  unsigned h = hash_bits(key, LTB);
  for (int probe = 0; probe < LT; ++probe) {
    const unsigned long long k = ((volatile unsigned long long*)t.key)[h];
    if (k == key) return (int)h;
    if (k == EMPTY_KEY) {
      const unsigned f = atomicAdd(&t.fill, 1u);
      if (f + 1u >= LocalTable<LTB>::CAP) filled = true;
      if (f >= LocalTable<LTB>::CAP) return -1;
      const unsigned long long old = atomicCAS(&t.key[h], EMPTY_KEY, key);
      if (old == EMPTY_KEY) {
        created = true;
        return (int)h;
      }
      if (old == key) return (int)h;
    }
    h = (h + 1u) & (LT - 1u);
  }
  return -1;
}

// Merge the block's counters into the global table and zero them; with
// clear_keys the cells themselves are dropped as well (table full).
template <int LTB>
__device__ __forceinline__ void local_flush(LocalTable<LTB>& t, const StepBuffers& b, bool clear_keys) {
  const size_t hcap = size_t(1) << b.hbits;
  for (unsigned j = threadIdx.x; j < (unsigned)LocalTable<LTB>::LT; j += blockDim.x) {
    if (t.key[j] == EMPTY_KEY) continue;
    const unsigned cnt = t.acc[0][j];
    if (cnt != 0u) {
      const unsigned g = t.gslot[j];
      atomicAdd(&b.hcnt[g], cnt);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const long long bias = c < 2 ? POS_BIAS : VAL_BIAS;
        const long long sum = (long long)t.acc[1 + 2 * c][j] + ((long long)t.acc[2 + 2 * c][j] << PIECE_BITS) -
                              (long long)cnt * bias;
        atomicAdd((unsigned long long*)&b.hsum[c * hcap + g], (unsigned long long)sum);
      }
#pragma unroll
      for (int a = 0; a < NACC; ++a) t.acc[a][j] = 0u;
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

// Threads per block of the propagate/bin kernel: 512 with the small cell
// table (two blocks per SM), 1024 with the large one (one block per SM).
template <int LTB>
struct PbShape {
  static constexpr int THREADS = LTB == 10 ? PB_THREADS : 2 * PB_THREADS;
  static constexpr int CHUNK = THREADS * PB_PER_THREAD;
};

// A streamed load of state or noise.  With the large table (224 KB of shared memory) almost none of
// the SM's unified L1 is left, and loads cached there throttled the kernel (lg_throttle stalls):
// they bypass L1 (cached in L2 only) in that variant.
template <int LTB>
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  return LTB == 12 ? __ldcg(p) : *p;
}

// i-th particle (0..3) of this thread in the chunk: four consecutive indices
// when the rows allow 16-byte vector access, otherwise strided by the block.
template <bool VEC, int THREADS>
__device__ __forceinline__ int64_t pb_index(int64_t base, int k) {
  return VEC ? base + 4 * threadIdx.x + k : base + (int64_t)k * THREADS + threadIdx.x;
}

// GATHER: the input particle set is st[., src_idx[i]] (deferred resampling: the
// previous step recorded its ancestors and left the gather to this read).
// GEN: the process noise is drawn here from the counter-based generator (ng)
// instead of read from nz (FP32 state only).
template <typename T, bool VEC, int LTB, bool GATHER = false, bool GEN = false>
__global__ void __launch_bounds__(PbShape<LTB>::THREADS, LTB == 10 ? 2 : 1)
k_prop_bin(StepBuffers b, const T* __restrict__ st, const T* __restrict__ nz, int64_t N, T h, long long hq,
           const int32_t* __restrict__ src_idx = nullptr, NoiseGen ng = NoiseGen{}) {
  constexpr int THR = PbShape<LTB>::THREADS;
  constexpr int CHUNK = PbShape<LTB>::CHUNK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LocalTable<LTB>& tab = *reinterpret_cast<LocalTable<LTB>*>(smem_raw);
  T* __restrict__ prop = static_cast<T*>(b.prop);
  const size_t hcap = size_t(1) << b.hbits;
  for (int j = threadIdx.x; j < LocalTable<LTB>::LT; j += blockDim.x) {
    tab.key[j] = EMPTY_KEY;
#pragma unroll
    for (int a = 0; a < NACC; ++a) tab.acc[a][j] = 0u;
  }
  if (threadIdx.x == 0) {
    tab.fill = 0u;
    tab.hot = 0u;
  }
  // anchors of vx, vy, I0: particle 0's input value in fixed point
  long long anc[3];
  const int64_t src0 = GATHER ? (int64_t)src_idx[0] : 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) anc[c] = to_fixed(st[(2 + c) * N + src0], Scales<T>::VAL);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) b.ctl->anchor[2 + c] = anc[c];
  }
  __syncthreads();
  const T half = T(0.5);
  const T lim = T(1073741823.0);  // 2^30 - 1
  const int64_t nchunks = (N + CHUNK - 1) / CHUNK;
  constexpr unsigned HOT_AT = SLOT_PARTICLES - (unsigned)CHUNK;
  for (int64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const int64_t base = chunk * CHUNK;
    T v[PB_PER_THREAD][5];
    if (VEC && base + CHUNK <= N) {
      // 16-byte loads and stores of four consecutive particles per component
      const int64_t i0 = base + 4 * threadIdx.x;
      float4 sv[5], nv[5];
      if (GATHER) {
        // the four particles' sources: nondecreasing indices (systematic resampling), so a warp's
        // reads stay within a few cache lines per component
        const int4 a4 = *reinterpret_cast<const int4*>(src_idx + i0);
        const float* sf = reinterpret_cast<const float*>(st);
#pragma unroll
        for (int c = 0; c < 5; ++c)
          sv[c] = make_float4(sf[c * N + a4.x], sf[c * N + a4.y], sf[c * N + a4.z], sf[c * N + a4.w]);
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c)
          sv[c] = ld_stream<LTB>(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(st) + c * N + i0));
      }
      if (!GEN) {
#pragma unroll
        for (int c = 0; c < 5; ++c)
          nv[c] = ld_stream<LTB>(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(nz) + c * N + i0));
      }
      const float* sp[5] = {&sv[0].x, &sv[1].x, &sv[2].x, &sv[3].x, &sv[4].x};
      const float* np[5] = {&nv[0].x, &nv[1].x, &nv[2].x, &nv[3].x, &nv[4].x};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float e[5];
        if (GEN) {
          ng_noise5(ng, i0 + k, e);  // drawn particle by particle: no array of all four's noise
        } else {
#pragma unroll
          for (int c = 0; c < 5; ++c) e[c] = np[c][k];
        }
        v[k][0] = (T)add_rn(add_rn(sp[0][k], sp[2][k]), e[0]);
        v[k][1] = (T)add_rn(add_rn(sp[1][k], sp[3][k]), e[1]);
        v[k][2] = (T)add_rn(sp[2][k], e[2]);
        v[k][3] = (T)add_rn(sp[3][k], e[3]);
        v[k][4] = (T)add_rn(sp[4][k], e[4]);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        float4 o = make_float4((float)v[0][c], (float)v[1][c], (float)v[2][c], (float)v[3][c]);
        *reinterpret_cast<float4*>(reinterpret_cast<float*>(prop) + c * N + i0) = o;
      }
    } else {
#pragma unroll
      for (int k = 0; k < PB_PER_THREAD; ++k) {
        const int64_t i = pb_index<false, THR>(base, k);
        if (i < N) {
          if (GEN)
            propagate1_gen(st, ng, N, i, v[k], GATHER ? src_idx : nullptr);
          else
            propagate1(st, nz, N, i, v[k], GATHER ? src_idx : nullptr);
#pragma unroll
          for (int c = 0; c < 5; ++c) prop[c * N + i] = v[k][c];
        }
      }
    }
    const bool vec_chunk = VEC && base + CHUNK <= N;
    // each particle is summed into its cell as soon as the cell is found: the cell's counters are
    // usable at once, and only its global slot (written by the thread that took the cell into the
    // table) waits for the barrier below, before the slots are stored.  ls: the cell's local slot,
    // -3 - its global slot (table full), or -2 (no particle)
    int ls[PB_PER_THREAD];
    bool flag = false;  // this thread filled the table or brought a cell's count to the flush mark
#pragma unroll
    for (int k = 0; k < PB_PER_THREAD; ++k) {
      const int64_t i = vec_chunk ? pb_index<true, THR>(base, k) : pb_index<false, THR>(base, k);
      ls[k] = -2;
      if (i >= N) continue;
      T fx = floor_t(div_rn(add_rn(v[k][0], half), h));
      T fy = floor_t(div_rn(add_rn(v[k][1], half), h));
      if (!(finite_state(v[k]) && abs_t(fx) < lim && abs_t(fy) < lim)) {
        raise_flag(b.ctl, PCSIR_DERR_RANGE);
        fx = T(0);
        fy = T(0);
        v[k][0] = T(0);
        v[k][1] = T(0);
      }
      const int bx = (int)fx, by = (int)fy;
      const unsigned long long key = pack_key(bx, by);
      bool created;
      int s = local_find_or_insert(tab, key, created, flag);
      if (created) tab.gslot[s] = global_find_or_insert(b, key);
      long long bv[5];
      bv[0] = to_fixed(v[k][0], Scales<T>::POS) - (long long)bx * hq + POS_BIAS;
      bv[1] = to_fixed(v[k][1], Scales<T>::POS) - (long long)by * hq + POS_BIAS;
#pragma unroll
      for (int c = 0; c < 3; ++c) bv[2 + c] = to_fixed(v[k][2 + c], Scales<T>::VAL) - anc[c] + VAL_BIAS;
      bool bad = false;
#pragma unroll
      for (int c = 0; c < 5; ++c) bad |= (bv[c] < 0 || bv[c] >= BIASED_LIMIT);
      if (bad) {
        raise_flag(b.ctl, PCSIR_DERR_RANGE);
        bv[0] = bv[1] = POS_BIAS;
        bv[2] = bv[3] = bv[4] = VAL_BIAS;
      }
      if (s >= 0) {
        if (atomicAdd(&tab.acc[0][s], 1u) + 1u == HOT_AT) {
          tab.hot = 1u;
          flag = true;
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          atomicAdd(&tab.acc[1 + 2 * c][s], (unsigned)(bv[c] & PIECE_MASK));
          atomicAdd(&tab.acc[2 + 2 * c][s], (unsigned)(bv[c] >> PIECE_BITS));
        }
      } else {
        const unsigned g = global_find_or_insert(b, key);
        atomicAdd(&b.hcnt[g], 1u);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const long long bias = c < 2 ? POS_BIAS : VAL_BIAS;
          atomicAdd((unsigned long long*)&b.hsum[c * hcap + g], (unsigned long long)(bv[c] - bias));
        }
        s = -3 - (int)g;
      }
      ls[k] = s;
    }
    // the table is flushed after this chunk when some thread filled it or raised a cell to the
    // flush mark: every thread learns it from this barrier itself, so none reads the table's
    // counters while another may already be inserting the next chunk's cells
    const bool flush = __syncthreads_or(flag) != 0;
    {
      // the particles' global slots: a cell taken into the table during this chunk has its slot
      // written before the barrier; the table's next changes (a flush, new cells in empty slots)
      // touch no slot read here
      unsigned gs[PB_PER_THREAD];
#pragma unroll
      for (int k = 0; k < PB_PER_THREAD; ++k)
        gs[k] = ls[k] >= 0 ? tab.gslot[ls[k]] : (ls[k] == -2 ? 0u : (unsigned)(-3 - ls[k]));
      if (vec_chunk) {
        *reinterpret_cast<uint4*>(b.pslot + base + 4 * threadIdx.x) = make_uint4(gs[0], gs[1], gs[2], gs[3]);
      } else {
#pragma unroll
        for (int k = 0; k < PB_PER_THREAD; ++k)
          if (ls[k] != -2) b.pslot[pb_index<false, THR>(base, k)] = gs[k];
      }
    }
    if (flush) local_flush(tab, b, tab.fill >= LocalTable<LTB>::CAP);  // read before the flush's first barrier
  }
  local_flush(tab, b, false);
}

// ---------------------------------------------------------------------------
// Dummies and their likelihood (Algorithm 2: mean state of each bin, weight
// update of the dummy only).  One warp per occupied bin.
// ---------------------------------------------------------------------------
constexpr int BIN_THREADS = 256;
constexpr int MAXP = 127;  // largest patch side (shared-memory factor tables)

__device__ __forceinline__ void block_max_to_global(double v, Control* ctl) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = -INFINITY;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) m = fmax(m, red[j]);
    if (m > -INFINITY) atomicMax(&ctl->max_ll, ord_encode(m));
  }
}

// threads evaluating one dummy: a warp, the same partition as the per-particle
// SIR kernel, so a bin holding a single particle gives SIR's value bit for bit
constexpr int BIN_GROUP = 32;

__device__ __forceinline__ void block_max_llq_to_global(long long v, Control* ctl) {
  __shared__ long long red[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = LLQ_NONE;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) m = red[j] > m ? red[j] : m;
    if (m != LLQ_NONE) atomicMax(&ctl->max_llq, llq_enc(m));
  }
}

// With SUR (a likelihood surrogate is attached) the exact likelihood is
// evaluated only for dummies whose surrogate patch leaves the image (their
// value is final) and for held-out dummies (their value goes to the held-out
// list, and the surrogate's prediction to bin_ll).
struct SurBins {
  unsigned long long salt;
  double frac;
  int min_holdout;
  int ho_cap;
  int* ho_bin;
  double* ho_ll;
  SurStats* stats;
};

template <bool SUR>
__global__ void __launch_bounds__(BIN_THREADS)
k_bins(StepBuffers b, LikParams lp, const float* __restrict__ img, int W, int H, long long hq, double h, int coc,
       SurBins sb) {
  constexpr int NG = BIN_THREADS / BIN_GROUP;
  __shared__ float scratch[NG][4 * MAXP];
  __shared__ int red[NG][3 * (BIN_GROUP / 32)];
  const int group = threadIdx.x / BIN_GROUP, gtid = threadIdx.x % BIN_GROUP;
  const unsigned B = b.ctl->nocc;
  const size_t hcap = size_t(1) << b.hbits;
  const int64_t bs = b.bin_stride;
  const unsigned thr = SUR ? sur_holdout_threshold(sb.frac, sb.min_holdout, B) : 0u;
  double mymax = -INFINITY;
  for (unsigned bi = blockIdx.x * NG + group; bi < B; bi += gridDim.x * NG) {
    const unsigned g = b.occ[bi];
    const unsigned long long key = b.hkey[g];
    const int bx = key_bx(key), by = key_by(key);
    const unsigned n = b.hcnt[g];
    const double dn = (double)n;
    const double rdn = 1.0 / dn;  // one FP64 division per cell (GB300's FP64 rate is low)
    double mean[5];
    mean[0] = ((double)((long long)bx * hq) + (double)b.hsum[g] * rdn) * POS_INV;
    mean[1] = ((double)((long long)by * hq) + (double)b.hsum[hcap + g] * rdn) * POS_INV;
#pragma unroll
    for (int c = 2; c < 5; ++c) mean[c] = ((double)b.ctl->anchor[c] + (double)b.hsum[c * hcap + g] * rdn) * VAL_INV;
    if (coc) {  // pcSIR-CoC: the cell's geometric centre
      mean[0] = ((double)bx + 0.5) * h - 0.5;
      mean[1] = ((double)by + 0.5) * h - 0.5;
    }
    if (gtid == 0) {
      b.bin_xy[bi] = bx;
      b.bin_xy[bs + bi] = by;
      b.bin_cnt[bi] = n;
#pragma unroll
      for (int c = 0; c < 5; ++c) b.dummy[c * bs + bi] = mean[c];
      b.hrank[g] = bi;
    }
    bool clipped = false, held = false;
    if (SUR) {
      int cx, cy;
      clipped = !sur_origin(mean[0], mean[1], W, H, &cx, &cy);
      held = !clipped && sur_held(bx, by, sb.salt, thr);
      if (!clipped && !held) continue;  // uniform over the group: the surrogate predicts this dummy
    }
    double ll = ll_to_double(group_loglik<BIN_GROUP>(img, W, H, lik_pos(mean[0], mean[1], mean[4]), lp,
                                                     scratch[group], red[group], group, gtid));
    if (!isfinite(ll)) {
      if (gtid == 0) raise_flag(b.ctl, PCSIR_DERR_NONFINITE);
      ll = -INFINITY;
    }
    if (SUR && held) {
      if (gtid == 0) {
        const unsigned slot = atomicAdd(&sb.stats->n_ho, 1u);
        if (slot < (unsigned)sb.ho_cap) {
          sb.ho_bin[slot] = (int)bi;
          sb.ho_ll[slot] = ll;
        }
      }
      continue;
    }
    if (SUR && gtid == 0) atomicAdd(&sb.stats->n_clipped, 1u);
    if (gtid == 0) b.bin_ll[bi] = ll;
    mymax = fmax(mymax, ll);
  }
  block_max_to_global(mymax, b.ctl);
}

// Exact likelihood of every dummy when the held-out check rejected the
// surrogate's predictions (stats->fallback); otherwise returns at once.  The
// dummy states are those k_bins stored, so the values equal the plain step's.
__global__ void __launch_bounds__(BIN_THREADS)
k_bins_fallback(StepBuffers b, LikParams lp, const float* __restrict__ img, int W, int H,
                const SurStats* __restrict__ stats) {
  if (*(volatile const unsigned*)&stats->fallback == 0u) return;
  constexpr int NG = BIN_THREADS / BIN_GROUP;
  __shared__ float scratch[NG][4 * MAXP];
  __shared__ int red[NG][3 * (BIN_GROUP / 32)];
  const int group = threadIdx.x / BIN_GROUP, gtid = threadIdx.x % BIN_GROUP;
  const unsigned B = b.ctl->nocc;
  const int64_t bs = b.bin_stride;
  double mymax = -INFINITY;
  for (unsigned bi = blockIdx.x * NG + group; bi < B; bi += gridDim.x * NG) {
    const double x = b.dummy[bi], y = b.dummy[bs + bi], a = b.dummy[4 * bs + bi];
    double ll = ll_to_double(group_loglik<BIN_GROUP>(img, W, H, lik_pos(x, y, a), lp, scratch[group], red[group],
                                                     group, gtid));
    if (!isfinite(ll)) {
      if (gtid == 0) raise_flag(b.ctl, PCSIR_DERR_NONFINITE);
      ll = -INFINITY;
    }
    if (gtid == 0) b.bin_ll[bi] = ll;
    mymax = fmax(mymax, ll);
  }
  block_max_to_global(mymax, b.ctl);
}

// ---------------------------------------------------------------------------
// Weight reductions.  w~ = exp(ll - max) per bin (pcSIR) or per particle
// (SIR); integer weights q = rint(w~ 2^sq) for the exact scan; sums for the
// normaliser, the ESS and the posterior mean.  The last block to finish
// writes the step's scalar results.
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;

struct RedAcc {
  double Tf, T2, est[5];
  long long Tint;
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// nblocks: the number of blocks taking part (the last of them writes the results)
__device__ void block_reduce_commit(RedAcc a, const StepBuffers& b, int64_t N, int kind, bool with_est,
                                    unsigned nblocks) {
  __shared__ double sd[7][RED_THREADS / 32];
  __shared__ long long sl[RED_THREADS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double vals[7] = {a.Tf, a.T2, a.est[0], a.est[1], a.est[2], a.est[3], a.est[4]};
#pragma unroll
  for (int k = 0; k < 7; ++k) vals[k] = warp_sum_d(vals[k]);
  const long long ti = warp_sum_ll(a.Tint);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 7; ++k) sd[k][w] = vals[k];
    sl[w] = ti;
  }
  __syncthreads();
  Control* ctl = b.ctl;
  if (threadIdx.x == 0) {
    double t[7] = {0, 0, 0, 0, 0, 0, 0};
    long long tt = 0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) {
#pragma unroll
      for (int k = 0; k < 7; ++k) t[k] += sd[k][j];
      tt += sl[j];
    }
    atomicAdd(&ctl->T_f, t[0]);
    atomicAdd(&ctl->T2_f, t[1]);
    if (with_est) {
#pragma unroll
      for (int c = 0; c < 5; ++c) atomicAdd(&ctl->est[c], t[2 + c]);
    }
    atomicAdd((unsigned long long*)&ctl->T_int, (unsigned long long)tt);
    __threadfence();
    last = (atomicAdd(&ctl->done_blocks, 1u) == nblocks - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    volatile Control* vc = ctl;
    const double Tf = vc->T_f, T2 = vc->T2_f;
    pcsir_result* r = b.dres;
    for (int c = 0; c < 5; ++c) r->estimate[c] = with_est ? vc->est[c] / Tf : 0.0;
    r->ess = Tf * Tf / T2;
    // kind 1: pcSIR (maximum over the dummies), 0: SIR, 2: pcSIR with per-particle
    // log-weights (both: maximum over the particles' fixed-point log-weights)
    if (kind == 1) {
      r->max_loglik = ord_decode(vc->max_ll);
    } else {
      const unsigned long long e = vc->max_llq;
      r->max_loglik = e == 0ull ? -INFINITY : (double)llq_dec(e) * (1.0 / 4294967296.0);
    }
    r->sum_wtilde = Tf;
    r->n_particles = N;
    r->n_bins = kind != 0 ? (int64_t)vc->nocc : 0;
    r->kind = kind != 0 ? 1 : 0;
    if (vc->T_int <= 0) atomicOr(&ctl->err, (unsigned)PCSIR_DERR_ZEROSUM);
  }
}

// The posterior mean (Alg. 1) is the weighted mean over particles: per bin,
// weight x member count x centre of mass.  With pcSIR-CoC the dummy sits at
// the cell centre, so the centre of mass of the position is recomputed from
// the exact sums here.
__global__ void __launch_bounds__(RED_THREADS) k_binred(StepBuffers b, int64_t N, int sq, long long hq, int coc) {
  const unsigned B = b.ctl->nocc;
  // only as many blocks as there are bins to cover take part
  const unsigned need = (B + blockDim.x - 1) / blockDim.x;
  const unsigned active = need < 1u ? 1u : (need < gridDim.x ? need : gridDim.x);
  if (blockIdx.x >= active) return;
  const double m = ord_decode(b.ctl->max_ll);
  const int64_t bs = b.bin_stride;
  RedAcc a = {0.0, 0.0, {0.0, 0.0, 0.0, 0.0, 0.0}, 0};
  const unsigned gstride = gridDim.x * blockDim.x;
  for (unsigned bi = blockIdx.x * blockDim.x + threadIdx.x; bi < B; bi += gstride) {
    const unsigned g = b.occ[bi];
    const double n = (double)b.bin_cnt[bi];
    const double ll = b.bin_ll[bi];
    const double wt = (ll == -INFINITY) ? 0.0 : exp(ll - m);
    const long long q = __double2ll_rn(ldexp(wt, sq));
    b.hq[g] = q;
    b.hw[g] = wt;
    a.Tf += n * wt;
    a.T2 += n * wt * wt;
    a.Tint += (long long)b.bin_cnt[bi] * q;
    double pos[2] = {b.dummy[bi], b.dummy[bs + bi]};
    if (coc) {
      const size_t hcap = size_t(1) << b.hbits;
      const unsigned long long key = b.hkey[g];
      pos[0] = ((double)((long long)key_bx(key) * hq) + (double)b.hsum[g] / n) * POS_INV;
      pos[1] = ((double)((long long)key_by(key) * hq) + (double)b.hsum[hcap + g] / n) * POS_INV;
    }
    a.est[0] += n * wt * pos[0];
    a.est[1] += n * wt * pos[1];
#pragma unroll
    for (int c = 2; c < 5; ++c) a.est[c] += n * wt * b.dummy[c * bs + bi];
  }
  block_reduce_commit(a, b, N, 1, true, active);
}

// ---------------------------------------------------------------------------
// SIR: propagate and evaluate the likelihood of every particle.
// ---------------------------------------------------------------------------
constexpr int SL_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(SL_THREADS)
k_sir_prop_lik(StepBuffers b, const T* __restrict__ st, const T* __restrict__ nz, int64_t N, LikParams lp,
               const float* __restrict__ img, int W, int H, int keep) {
  __shared__ T sx[SL_THREADS], sy[SL_THREADS], si[SL_THREADS];
  __shared__ float scratch[SL_THREADS / 32][4 * MAXP];
  T* __restrict__ prop = static_cast<T*>(b.prop);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * SL_THREADS;
  const int64_t i = base + threadIdx.x;
  if (i < N) {
    T v[5];
    propagate1(st, nz, N, i, v);
#pragma unroll
    for (int c = 0; c < 5; ++c) prop[c * N + i] = v[c];
    if (!finite_state(v)) {
      raise_flag(b.ctl, PCSIR_DERR_RANGE);
      v[0] = v[1] = v[4] = T(0);
    }
    sx[threadIdx.x] = v[0];
    sy[threadIdx.x] = v[1];
    si[threadIdx.x] = v[4];
  }
  __syncthreads();
  const int cnt = (int)((N - base) < SL_THREADS ? (N - base) : SL_THREADS);
  long long mymax = LLQ_NONE;
  for (int j = w; j < cnt; j += SL_THREADS / 32) {
    const LLSum ls = warp_loglik(img, W, H, lik_pos(sx[j], sy[j], si[j]), lp, scratch[w]);
    const long long q = llq_of(ls);
    if (lane == 0) {
      if (ls.bad) raise_flag(b.ctl, PCSIR_DERR_NONFINITE);
      b.llq[base + j] = q;
      if (keep & PCSIR_KEEP_LOGLIK) b.ll[base + j] = ll_to_double(ls);
    }
    mymax = q > mymax ? q : mymax;
  }
  block_max_llq_to_global(mymax, b.ctl);
}

// fixed-point log-likelihood of particle i: from the SIR kernel's array, or
// converted from a caller's float64 log-weight
__device__ __forceinline__ long long particle_llq(const long long* __restrict__ llq, int64_t i) { return llq[i]; }
__device__ __forceinline__ long long particle_llq(const double* __restrict__ lw, int64_t i) { return llq_of(lw[i]); }

template <typename T, typename SRC>
__global__ void __launch_bounds__(RED_THREADS) k_sir_w(StepBuffers b, const SRC* __restrict__ lls, int64_t N,
                                                       int sq, int with_est, int kind, long long* __restrict__ qout) {
  const unsigned long long me = b.ctl->max_llq;
  const long long mq = llq_dec(me);
  const T* __restrict__ prop = static_cast<const T*>(b.prop);
  kahan kt, k2, ke[5];
  long long tint = 0;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  // four of the thread's particles i, i + G, i + 2G, i + 3G per pass (G the grid's threads): their
  // loads and weights are formed together, then added in that order, as one at a time would
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < N; i0 += 4 * gstride) {
    df wd[4];
    float x[4][5];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + k * gstride;
      wd[k] = df{0.0f, 0.0f};
      if (i >= N) continue;
      if (me != 0ull) wd[k] = wtilde_q(particle_llq(lls, i), mq);
      if (with_est) {
#pragma unroll
        for (int c = 0; c < 5; ++c) x[k][c] = (float)prop[c * N + i];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + k * gstride;
      if (i >= N) continue;
      const float wt = wd[k].hi;
      const long long q = q_of_wtilde(wd[k], sq);
      tint += q;
      if (qout) qout[i] = q;  // the resampling reads the integer weights instead of forming them again
      kt.add(wt);
      k2.add(wt * wt);
      if (with_est) {
#pragma unroll
        for (int c = 0; c < 5; ++c) ke[c].add(wt * x[k][c]);
      }
    }
  }
  RedAcc a;
  a.Tf = (double)kt.s - (double)kt.c;
  a.T2 = (double)k2.s - (double)k2.c;
#pragma unroll
  for (int c = 0; c < 5; ++c) a.est[c] = (double)ke[c].s - (double)ke[c].c;
  a.Tint = tint;
  block_reduce_commit(a, b, N, kind, with_est != 0, gridDim.x);
}

// max of caller-given log-weights (standalone resampling)
__global__ void __launch_bounds__(RED_THREADS) k_logw_max(StepBuffers b, const double* __restrict__ lw, int64_t N) {
  long long m = LLQ_NONE;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gstride) {
    const long long v = llq_of(lw[i]);
    m = v > m ? v : m;
  }
  block_max_llq_to_global(m, b.ctl);
}

// ---------------------------------------------------------------------------
// Standalone likelihood of given positions: one warp per position.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BIN_THREADS)
k_loglik(LikParams lp, const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ a,
         int64_t n, const float* __restrict__ img, int W, int H, double* __restrict__ out) {
  __shared__ float scratch[BIN_THREADS / 32][4 * MAXP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t j = (int64_t)blockIdx.x * (BIN_THREADS / 32) + w; j < n; j += (int64_t)gridDim.x * (BIN_THREADS / 32)) {
    const double ll = ll_to_double(warp_loglik(img, W, H, lik_pos(x[j], y[j], a[j]), lp, scratch[w]));
    if (lane == 0) out[j] = ll;
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
LikParams make_lik(const ModelParams& m) {
  LikParams lp;
  lp.P = m.P;
  lp.kind = m.kind;
  lp.bg = (float)m.bg;
  const double c2 = 1.0 / (2.0 * m.sigma * m.sigma);
  lp.c2.hi = (float)c2;
  lp.c2.lo = (float)(c2 - (double)lp.c2.hi);
  lp.inv2sxi2 = (float)(1.0 / (2.0 * m.sigma_xi * m.sigma_xi));
  return lp;
}

int weight_scale_bits(int64_t N) {
  int lg = 0;
  while ((int64_t(1) << lg) < N) ++lg;
  return 61 - lg;
}

// One-time kernel attributes and occupancy, queried at context creation so
// that step calls only enqueue work (and stay legal inside a stream capture).
template <typename K>
static cudaError_t prop_bin_attr(K kern, size_t smem, int threads, int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int g = 1;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g, kern, threads, smem);
  if (g < *per_sm) *per_sm = g;
  return e;
}

template <typename T, bool VEC, int LTB>
static cudaError_t prop_bin_prepare1(int* per_sm) {
  const size_t smem = sizeof(LocalTable<LTB>);
  constexpr int THR = PbShape<LTB>::THREADS;
  // the grid is sized for the variant that fits the fewest blocks per SM
  *per_sm = 1 << 20;
  cudaError_t e = prop_bin_attr(k_prop_bin<T, VEC, LTB>, smem, THR, per_sm);
  if (e == cudaSuccess) e = prop_bin_attr(k_prop_bin<T, VEC, LTB, true>, smem, THR, per_sm);
  if (std::is_same<T, float>::value) {
    if (e == cudaSuccess) e = prop_bin_attr(k_prop_bin<T, VEC, LTB, false, true>, smem, THR, per_sm);
    if (e == cudaSuccess) e = prop_bin_attr(k_prop_bin<T, VEC, LTB, true, true>, smem, THR, per_sm);
  }
  if (*per_sm < 1) *per_sm = 1;
  return e;
}

template <int LTB>
static cudaError_t prop_bin_prepare(int dtype, int* per_sm) {
  int a = 1, c = 1;
  cudaError_t e;
  if (dtype == PCSIR_F32) {
    e = prop_bin_prepare1<float, true, LTB>(&a);
    if (e == cudaSuccess) e = prop_bin_prepare1<float, false, LTB>(&c);
  } else {
    e = prop_bin_prepare1<double, false, LTB>(&a);
    c = a;
  }
  *per_sm = a < c ? a : c;
  return e;
}

cudaError_t prepare_kernels(int dtype, int* prop_bin_per_sm) {
  cudaError_t e = prop_bin_prepare<10>(dtype, &prop_bin_per_sm[0]);
  if (e == cudaSuccess) e = prop_bin_prepare<12>(dtype, &prop_bin_per_sm[1]);
  return e;
}

template <typename T, int LTB>
static cudaError_t prop_bin_launch_t(const StepBuffers& b, const void* state, const void* noise, int64_t N, double h,
                                     int num_sms, int per_sm, cudaStream_t s, long long hq, const int32_t* src_idx,
                                     const NoiseGen* ng) {
  const size_t smem = sizeof(LocalTable<LTB>);
  constexpr int THR = PbShape<LTB>::THREADS;
  const int64_t nchunks = (N + PbShape<LTB>::CHUNK - 1) / PbShape<LTB>::CHUNK;
  const int grid = (int)std::min<int64_t>(nchunks, (int64_t)num_sms * per_sm);
  const bool vec = std::is_same<T, float>::value && (N % 4 == 0) &&
                   ((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(noise) |
                     reinterpret_cast<uintptr_t>(b.prop) | reinterpret_cast<uintptr_t>(b.pslot) |
                     reinterpret_cast<uintptr_t>(src_idx)) % 16 == 0);
  const T* st = static_cast<const T*>(state);
  const T* nz = static_cast<const T*>(noise);
  if (ng != nullptr) {
    if (!std::is_same<T, float>::value) return cudaErrorInvalidValue;  // FP32 state only
    const bool vg = std::is_same<T, float>::value && (N % 4 == 0) &&
                    ((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(b.prop) |
                      reinterpret_cast<uintptr_t>(b.pslot) | reinterpret_cast<uintptr_t>(src_idx)) % 16 == 0);
    if (src_idx != nullptr) {
      if (vg)
        k_prop_bin<T, true, LTB, true, true><<<grid, THR, smem, s>>>(b, st, nullptr, N, (T)h, hq, src_idx, *ng);
      else
        k_prop_bin<T, false, LTB, true, true><<<grid, THR, smem, s>>>(b, st, nullptr, N, (T)h, hq, src_idx, *ng);
    } else if (vg) {
      k_prop_bin<T, true, LTB, false, true><<<grid, THR, smem, s>>>(b, st, nullptr, N, (T)h, hq, nullptr, *ng);
    } else {
      k_prop_bin<T, false, LTB, false, true><<<grid, THR, smem, s>>>(b, st, nullptr, N, (T)h, hq, nullptr, *ng);
    }
    return cudaGetLastError();
  }
  if (src_idx != nullptr) {
    if (vec)
      k_prop_bin<T, true, LTB, true><<<grid, THR, smem, s>>>(b, st, nz, N, (T)h, hq, src_idx);
    else
      k_prop_bin<T, false, LTB, true><<<grid, THR, smem, s>>>(b, st, nz, N, (T)h, hq, src_idx);
  } else if (vec) {
    k_prop_bin<T, true, LTB><<<grid, THR, smem, s>>>(b, st, nz, N, (T)h, hq);
  } else {
    k_prop_bin<T, false, LTB><<<grid, THR, smem, s>>>(b, st, nz, N, (T)h, hq);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t prop_bin_launch(const StepBuffers& b, const void* state, const void* noise, int64_t N, double h,
                                   int num_sms, cudaStream_t s, long long hq, const int32_t* src_idx,
                                   const NoiseGen* ng = nullptr) {
  if (b.big_table)
    return prop_bin_launch_t<T, 12>(b, state, noise, N, h, num_sms, b.prop_bin_per_sm[1], s, hq, src_idx, ng);
  return prop_bin_launch_t<T, 10>(b, state, noise, N, h, num_sms, b.prop_bin_per_sm[0], s, hq, src_idx, ng);
}

static cudaError_t mark(StageEvents se, int j, cudaStream_t s) {
  return se.ev ? cudaEventRecord(se.ev[j], s) : cudaSuccess;
}

cudaError_t launch_pcsir_front(const StepBuffers& b, const ModelParams& m, int dtype, const void* state,
                               const void* noise, int64_t N, double h, const float* img, int W, int H,
                               int num_sms, cudaStream_t s, StageEvents se, const SurStep* sur,
                               const int32_t* src_idx, const NoiseGen* ng) {
  const long long hq = llrint(h * 2147483648.0);
  cudaError_t e = dtype == PCSIR_F32 ? prop_bin_launch<float>(b, state, noise, N, h, num_sms, s, hq, src_idx, ng)
                                     : prop_bin_launch<double>(b, state, noise, N, h, num_sms, s, hq, src_idx, ng);
  if (e != cudaSuccess || (e = mark(se, 1, s)) != cudaSuccess) return e;
  const LikParams lp = make_lik(m);
  if (sur == nullptr) {
    k_bins<false><<<num_sms * 4, BIN_THREADS, 0, s>>>(b, lp, img, W, H, hq, h, m.coc, SurBins{});
    e = cudaGetLastError();
  } else {
    const SurBins sb{sur->salt, sur->frac, sur->min_holdout, sur->ho_cap, sur->ho_bin, sur->ho_ll, sur->stats};
    k_bins<true><<<num_sms * 4, BIN_THREADS, 0, s>>>(b, lp, img, W, H, hq, h, m.coc, sb);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_sur_step(*sur, b, m, img, W, H, s);
    if (e == cudaSuccess) {
      k_bins_fallback<<<num_sms * 4, BIN_THREADS, 0, s>>>(b, lp, img, W, H, sur->stats);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess || (e = mark(se, 2, s)) != cudaSuccess) return e;
  k_binred<<<num_sms * 2, RED_THREADS, 0, s>>>(b, N, weight_scale_bits(N), hq, m.coc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return mark(se, 3, s);
}

cudaError_t launch_sir_front(const StepBuffers& b, const ModelParams& m, int dtype, const void* state,
                             const void* noise, int64_t N, const float* img, int W, int H, int num_sms,
                             cudaStream_t s, StageEvents se, int keep, int with_weights) {
  const LikParams lp = make_lik(m);
  const int64_t nb = (N + SL_THREADS - 1) / SL_THREADS;
  const int sq = weight_scale_bits(N);
  const int rgrid = (int)std::min<int64_t>((N + RED_THREADS - 1) / RED_THREADS, (int64_t)num_sms * 4);
  if (dtype == PCSIR_F32) {
    k_sir_prop_lik<float><<<(unsigned)nb, SL_THREADS, 0, s>>>(b, static_cast<const float*>(state),
                                                             static_cast<const float*>(noise), N, lp, img, W, H,
                                                             keep);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || (e = mark(se, 1, s)) != cudaSuccess) return e;
    if (with_weights) k_sir_w<float, long long><<<rgrid, RED_THREADS, 0, s>>>(b, b.llq, N, sq, 1, 0, nullptr);
  } else {
    k_sir_prop_lik<double><<<(unsigned)nb, SL_THREADS, 0, s>>>(b, static_cast<const double*>(state),
                                                              static_cast<const double*>(noise), N, lp, img, W, H,
                                                              keep);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || (e = mark(se, 1, s)) != cudaSuccess) return e;
    if (with_weights) k_sir_w<double, long long><<<rgrid, RED_THREADS, 0, s>>>(b, b.llq, N, sq, 1, 0, nullptr);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || (e = mark(se, 2, s)) != cudaSuccess) return e;
  return mark(se, 3, s);
}

cudaError_t launch_logw_front(const StepBuffers& b, const double* logw, int64_t N, int num_sms, cudaStream_t s) {
  const int rgrid = (int)std::min<int64_t>((N + RED_THREADS - 1) / RED_THREADS, (int64_t)num_sms * 4);
  k_logw_max<<<rgrid, RED_THREADS, 0, s>>>(b, logw, N);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sir_w<float, double><<<rgrid, RED_THREADS, 0, s>>>(b, logw, N, weight_scale_bits(N), 0, 0, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_prop_bin(const StepBuffers& b, int dtype, const void* state, const void* noise, int64_t N,
                            double h, int num_sms, cudaStream_t s) {
  const long long hq = llrint(h * 2147483648.0);
  return dtype == PCSIR_F32 ? prop_bin_launch<float>(b, state, noise, N, h, num_sms, s, hq, nullptr)
                            : prop_bin_launch<double>(b, state, noise, N, h, num_sms, s, hq, nullptr);
}

// The resampled particle set written out: out[., i] = src[., idx[i]] (idx == nullptr: a copy).
template <typename T>
__global__ void __launch_bounds__(256) k_gather_state(const T* __restrict__ src, const int32_t* __restrict__ idx,
                                                      T* __restrict__ out, int64_t N) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx ? (int64_t)idx[i] : i;
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c * N + i] = src[c * N + j];
  }
}

cudaError_t launch_gather_state(int dtype, const void* src, const int32_t* idx, void* out, int64_t N,
                                cudaStream_t s) {
  const int64_t want = (N + 255) / 256;
  const unsigned grid = (unsigned)(want < (1 << 20) ? want : (1 << 20));
  if (dtype == PCSIR_F32)
    k_gather_state<float><<<grid, 256, 0, s>>>(static_cast<const float*>(src), idx, static_cast<float*>(out), N);
  else
    k_gather_state<double><<<grid, 256, 0, s>>>(static_cast<const double*>(src), idx, static_cast<double*>(out), N);
  return cudaGetLastError();
}

cudaError_t launch_particle_weights(const StepBuffers& b, int dtype, int64_t N, int num_sms, int kind,
                                    cudaStream_t s) {
  const int rgrid = (int)std::min<int64_t>((N + RED_THREADS - 1) / RED_THREADS, (int64_t)num_sms * 4);
  const int sq = weight_scale_bits(N);
  // the per-particle integer weights go to b.hq (capacity >= 2 N), read by WSRC_Q resampling
  if (dtype == PCSIR_F32)
    k_sir_w<float, long long><<<rgrid, RED_THREADS, 0, s>>>(b, b.llq, N, sq, 1, kind, b.hq);
  else
    k_sir_w<double, long long><<<rgrid, RED_THREADS, 0, s>>>(b, b.llq, N, sq, 1, kind, b.hq);
  return cudaGetLastError();
}

cudaError_t launch_loglik(const ModelParams& m, const double* x, const double* y, const double* i0, int64_t n,
                          const float* img, int W, int H, double* out, int num_sms, cudaStream_t s) {
  const LikParams lp = make_lik(m);
  const int64_t want = (n + (BIN_THREADS / 32) - 1) / (BIN_THREADS / 32);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 8));
  k_loglik<<<grid, BIN_THREADS, 0, s>>>(lp, x, y, i0, n, img, W, H, out);
  return cudaGetLastError();
}

}  // namespace pcsir
