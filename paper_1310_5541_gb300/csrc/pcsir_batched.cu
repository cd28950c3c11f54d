// Batched multi-target pcSIR: many independent targets (each its own
// Algorithm 2 filter, with its own particle count, PSF, patch and cell edge)
// advance by one step in a single persistent cooperative launch.  The phases
//   A  propagate + cell + centre-of-mass sums (cells keyed by target),
//   B  dummies and their likelihood,
//   C  per-target weights, normaliser, ESS, posterior mean,
//   D  per-(target, tile) sums of the integer weights,
//   E  per-target scan of its tile sums and the 64.64 resampling map,
//   F  per-(target, tile) systematic resampling and state gather
// are separated by grid-wide barriers whose waits are bounded: a wait that
// runs out sets PCSIR_DERR_TIMEOUT and every block leaves the kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pcsir_device.cuh"

namespace pcsir {

struct BatchTarget {
  long long off;     // first particle of the target in the concatenated arrays
  long long n;       // particles of the target
  long long hq;      // cell edge in units of 2^-31 px
  double h;          // cell edge (px)
  double sigma;      // PSF std
  float bg;          // background
  int patch;         // odd patch side
  int sq;            // integer-weight scale bits (n 2^sq <= 2^61)
  int tile0;         // first global tile of the target
  int ntiles;        // tiles of the target
  float hf;          // cell edge as float (the per-particle cell index; a double here would cost an
                     // FP64-pipe conversion per particle)
  df c2;             // 1 / (2 sigma^2) as double-float
};

struct BatchStats {  // per target, zeroed every step
  unsigned long long max_ll;
  long long T_int;
  double T_f, T2_f, est[5];
  unsigned long long dhi, dlo, uhi, ulo;
  long long anchor[3];
  unsigned int nbins;
  float inv_delta;  // 1 / Delta rounded to FP32 (first guesses of output indices)
};

struct BatchCtl {  // zeroed every step
  unsigned int nocc;
  unsigned int err;
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned int abort;
  unsigned int chunk_next;  // propagation phase: the next chunk to hand out
  unsigned long long phase_ns[8];  // global-timer reading of block 0 at the start and after each phase
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// block 0, thread 0 stamps the moment it passes phase boundary k
__device__ __forceinline__ void stamp(BatchCtl* c, int k) {
  if (blockIdx.x == 0 && threadIdx.x == 0) c->phase_ns[k] = global_ns();
}

struct BatchBufs {
  const BatchTarget* tg;
  BatchStats* st;
  BatchCtl* ctl;
  const long long* offs;  // [T + 1]
  int T;
  int ntiles_total;
  long long ntot;
  // hash table over (target, cell)
  unsigned long long* hkey;
  unsigned int* hcnt;
  long long* hsum;
  long long* hq;
  int hbits;
  unsigned int* occ;
  double* bin_ll;
  unsigned int* bin_cnt;
  unsigned long long* bin_key;
  unsigned int* pslot;
  float* prop;           // [5][pstride] propagated states
  long long pstride;     // row stride of prop: ntot rounded up to a multiple of 4
  long long* tile_sum;
  long long* tile_excl;
  const int* tile_target;  // [ntiles_total] target owning each tile (fixed at creation)
  int lik_group;           // lanes per cell in the likelihood phase: 8 (patches <= 15), 16 (<= 31) or 32
  pcsir_result* res;  // [T]
  // optional per-particle outputs (nullptr unless kept): target-local ancestor of every output
  // particle and the integer weight of every propagated particle
  int* anc;
  long long* qout;
  // set when a barrier wait ran out: the cell table may hold a partial step, and the next step
  // clears it before use (persists across steps; zeroed at creation)
  unsigned int* dirty;
  int bar_spins;  // polls of each barrier wait before it gives up
  int bar_fail;   // index of a barrier made unreachable (its wait runs out), -1 = none
  // deferred resampling (pcsir_batched_deferred_step), nullptr in a plain step: the step's input
  // state of particle i is gsrc[c pstride + ganc[i]] (the previous step's propagated states
  // through its ancestors, global indices), and the resampling phase writes each output's
  // ancestor to ganc instead of moving the states
  const float* gsrc;
  int* ganc;
};

constexpr int BT_THREADS = 512;
constexpr int BT_PER_THREAD = 4;
constexpr int BT_CHUNK = BT_THREADS * BT_PER_THREAD;
constexpr long long BT_GRAB_MAX = 16;  // longest run of chunks a block takes at once (propagation phase)
// the block-private cell table has 2^LTB slots (a kernel variant per LTB, chosen at run time by
// the autotuner) and takes new cells until three quarters of them are used
constexpr int BT_LTB_DEFAULT = 10;
constexpr int BT_LTB_MIN = 9, BT_LTB_MAX = 11;
constexpr int BT_PIECE_BITS = 18;
constexpr unsigned BT_PIECE_MASK = (1u << BT_PIECE_BITS) - 1u;
// a slot's 32-bit counters hold the pieces (< 2^18) of at most 2^14 particles; the table is
// flushed after any chunk that leaves some slot at 2^14 - BT_CHUNK particles or more
constexpr unsigned BT_HOT_AT = (1u << 14) - (unsigned)BT_CHUNK;
constexpr long long BT_POS_BIAS = 1ll << 33;
constexpr long long BT_VAL_BIAS = 1ll << 34;
constexpr long long BT_BIASED_LIMIT = 1ll << 36;
constexpr int BT_NACC = 11;
constexpr int BT_MAX_TARGETS = 2047;
constexpr int BT_TILE = 4096;
constexpr int BT_ITEMS = BT_TILE / BT_THREADS;  // 8
constexpr int BT_BARRIER_SPINS = 1 << 22;
constexpr int BT_NBARRIERS = 7;  // barriers 0 .. 6 of k_batched_step

// cell key: target (11 bits) | by + 2^25 (26 bits) | bx + 2^25 (26 bits)
__device__ __forceinline__ unsigned long long bkey(int t, int bx, int by) {
  return ((unsigned long long)t << 52) | ((unsigned long long)(unsigned)(by + (1 << 25)) << 26) |
         (unsigned long long)(unsigned)(bx + (1 << 25));
}
__device__ __forceinline__ int bkey_t(unsigned long long k) { return (int)(k >> 52); }
__device__ __forceinline__ int bkey_by(unsigned long long k) { return (int)((k >> 26) & 0x3ffffffu) - (1 << 25); }
__device__ __forceinline__ int bkey_bx(unsigned long long k) { return (int)(k & 0x3ffffffu) - (1 << 25); }

template <int LTB>
struct BatchLocal {
  static constexpr int LT = 1 << LTB;
  static constexpr unsigned CAP = 3u << (LTB - 2);
  unsigned long long key[LT];
  unsigned int acc[BT_NACC][LT];
  unsigned int gslot[LT];
  unsigned short list[LT];
  unsigned int nlist;
  unsigned int fill;
  unsigned int hot;  // some slot may reach 2^14 particles within the next chunk: flush
};

struct BatchResampleSmem {
  long long Cs[BT_TILE + BT_TILE / 16];  // inclusive cumulative integer weights, padded (j + j / 16)
  long long wtot[BT_THREADS / 32];
  long long s_lo, s_hi;
};

__host__ __device__ constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
template <int LTB>
__host__ __device__ constexpr size_t bt_smem_union() {
  return cmax(sizeof(BatchLocal<LTB>), sizeof(BatchResampleSmem));
}
template <int LTB>
constexpr size_t bt_smem() {
  return bt_smem_union<LTB>() + sizeof(long long) * (BT_MAX_TARGETS + 1);
}

// ---------------------------------------------------------------------------
// bounded grid-wide barrier (all blocks are co-resident: cooperative launch).  Barrier k
// releases when all gridDim.x blocks have arrived; the barrier b.bar_fail needs one arrival more
// than there are blocks, so that its wait runs out (a test of the timeout path).  A wait gives
// up after b.bar_spins polls: it raises PCSIR_DERR_TIMEOUT, the abort flag (every block then
// leaves at its next poll or barrier) and the dirty mark of the cell table.
// ---------------------------------------------------------------------------
__device__ __noinline__ bool grid_barrier(const BatchBufs& b, int k) {
  __shared__ unsigned s_ok;
  BatchCtl* c = b.ctl;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_ok = 1u;
    volatile BatchCtl* vc = c;
    const unsigned gen = vc->bar_gen;
    const unsigned need = gridDim.x + (k == b.bar_fail ? 1u : 0u);
    __threadfence();
    const unsigned arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == need - 1) {
      c->bar_count = 0u;
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      int spins = 0;
      while (vc->bar_gen == gen) {
        if (vc->abort) break;
        if (++spins > b.bar_spins) {
          atomicOr(&c->err, (unsigned)PCSIR_DERR_TIMEOUT);
          atomicExch(b.dirty, 1u);
          atomicExch(&c->abort, 1u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (vc->abort) s_ok = 0u;
  }
  __syncthreads();
  return s_ok != 0u;
}

__device__ unsigned bglobal_insert(const BatchBufs& b, unsigned long long key) {
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
  atomicOr(&b.ctl->err, (unsigned)PCSIR_DERR_RANGE);
  return 0;
}

// global slot of a cell the block's table has just taken: a chain of compare-and-swaps from slot h
// (the key's home slot, or the one after a first probe that met another key; a slot that holds the
// key or was empty and is now claimed ends it); created tells whether this call claimed the slot
__device__ unsigned bglobal_claim(const BatchBufs& b, unsigned long long key, bool& created, unsigned h) {
  const unsigned mask = (1u << b.hbits) - 1u;
  created = false;
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const unsigned long long old = atomicCAS(&b.hkey[h], EMPTY_KEY, key);
    if (old == EMPTY_KEY) {
      created = true;
      return h;
    }
    if (old == key) return h;
    h = (h + 1u) & mask;
  }
  atomicOr(&b.ctl->err, (unsigned)PCSIR_DERR_RANGE);
  return 0;
}

template <int LTB>
__device__ int blocal_insert(BatchLocal<LTB>& t, unsigned long long key, bool& created) {
  constexpr int LT = BatchLocal<LTB>::LT;
  created = false;
  unsigned h = hash_bits(key, LTB);
  for (int probe = 0; probe < LT; ++probe) {
    const unsigned long long k = ((volatile unsigned long long*)t.key)[h];
    if (k == key) return (int)h;
    if (k == EMPTY_KEY) {
      if (atomicAdd(&t.fill, 1u) >= BatchLocal<LTB>::CAP) return -1;
      const unsigned long long old = atomicCAS(&t.key[h], EMPTY_KEY, key);
      if (old == EMPTY_KEY) {
        created = true;
        t.list[atomicAdd(&t.nlist, 1u)] = (unsigned short)h;
        return (int)h;
      }
      if (old == key) return (int)h;
    }
    h = (h + 1u) & (LT - 1u);
  }
  return -1;
}

// Global slots of the cells that entered the block's table since list entry n0 (all of them,
// up to n1, after the chunk's insert pass): one claim chain per cell, all in parallel, and one
// append to the occupied list per warp.  Found inline by the inserting thread, a chunk that meets
// many new cells (many targets, small cells) waited on the thread with the most of them.
template <int LTB>
__device__ void blocal_resolve(BatchLocal<LTB>& t, const BatchBufs& b, unsigned n0, unsigned n1) {
  const unsigned lane = threadIdx.x & 31u;
  for (unsigned e0 = n0; e0 < n1; e0 += blockDim.x) {  // bound uniform over the block
    const unsigned e = e0 + threadIdx.x;
    bool created = false;
    unsigned g = 0u;
    if (e < n1) {
      const unsigned j = t.list[e];
      g = bglobal_claim(b, t.key[j], created, hash_bits(t.key[j], b.hbits));
      t.gslot[j] = g;
    }
    const unsigned m = __ballot_sync(0xffffffffu, created);
    if (m != 0u) {
      const unsigned leader = (unsigned)__ffs((int)m) - 1u;
      unsigned base = 0u;
      if (lane == leader) base = atomicAdd(&b.ctl->nocc, (unsigned)__popc((int)m));
      base = __shfl_sync(0xffffffffu, base, (int)leader);
      if (created) b.occ[base + (unsigned)__popc((int)(m & ((1u << lane) - 1u)))] = g;
    }
  }
}

template <int LTB>
__device__ void blocal_flush(BatchLocal<LTB>& t, const BatchBufs& b, bool clear_keys) {
  const size_t hcap = size_t(1) << b.hbits;
  const unsigned n = t.nlist;
  for (unsigned e = threadIdx.x; e < n; e += blockDim.x) {
    const unsigned j = t.list[e];
    const unsigned cnt = t.acc[0][j];
    if (cnt != 0u) {
      const unsigned g = t.gslot[j];
      atomicAdd(&b.hcnt[g], cnt);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const long long bias = c < 2 ? BT_POS_BIAS : BT_VAL_BIAS;
        const long long sum = (long long)t.acc[1 + 2 * c][j] + ((long long)t.acc[2 + 2 * c][j] << BT_PIECE_BITS) -
                              (long long)cnt * bias;
        atomicAdd((unsigned long long*)&b.hsum[c * hcap + g], (unsigned long long)sum);
      }
#pragma unroll
      for (int a = 0; a < BT_NACC; ++a) t.acc[a][j] = 0u;
    }
    if (clear_keys) t.key[j] = EMPTY_KEY;
  }
  __syncthreads();
  if (clear_keys && threadIdx.x == 0) {
    t.nlist = 0u;
    t.fill = 0u;
  }
  __syncthreads();
}

// the four floats starting m (0..3, uniform) elements after the 16-byte aligned quad a
__device__ __forceinline__ float4 shift_quad(const float4 a, const float4 b, int m) {
  switch (m) {
    case 0: return a;
    case 1: return make_float4(a.y, a.z, a.w, b.x);
    case 2: return make_float4(a.z, a.w, b.x, b.y);
    default: return make_float4(a.w, b.x, b.y, b.z);
  }
}

// target owning particle i (offsets in shared memory, T + 1 entries)
__device__ __forceinline__ int target_of(const long long* offs, int T, long long i) {
  int lo = 0, hi = T;  // offs[lo] <= i < offs[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (offs[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Phase A: propagate, cell, centre-of-mass sums (cf. k_prop_bin)
// ---------------------------------------------------------------------------
template <int LTB, bool DEF>
__device__ void phase_prop_bin(const BatchBufs& b, const float* __restrict__ st, const float* __restrict__ nz,
                               BatchLocal<LTB>& tab, const long long* offs) {
  const long long N = b.ntot;
  const long long P = b.pstride;
  const size_t hcap = size_t(1) << b.hbits;
  for (int j = threadIdx.x; j < BatchLocal<LTB>::LT; j += blockDim.x) {
    tab.key[j] = EMPTY_KEY;
#pragma unroll
    for (int a = 0; a < BT_NACC; ++a) tab.acc[a][j] = 0u;
  }
  if (threadIdx.x == 0) {
    tab.nlist = 0u;
    tab.fill = 0u;
    tab.hot = 0u;
  }
  __syncthreads();
  // each block takes runs of consecutive chunks from a shared counter, so that it meets the cells
  // of one or two targets at a time (a grid-stride order would show every block every target's
  // cells and overflow its table into per-particle global atomics), and a block slowed by many
  // cells takes fewer runs instead of holding up the phase.  The runs are guided: a run is the
  // remaining chunks over twice the grid, at most BT_GRAB_MAX, so that a block stays with a target
  // while much work is left and the last runs are single chunks (at 1000 targets and 22M
  // particles: a fixed range per block 0.75 ms, runs of two 0.66, guided runs 0.58, and with the
  // proactive flush below 0.55 ms)
  unsigned n_done = 0u, n_new = 0u;  // entries of tab.list whose global slot is known; cells new in the chunk
  const long long nchunks = (N + BT_CHUNK - 1) / BT_CHUNK;
  __shared__ long long s_grab, s_len;
  __shared__ bool s_clear;
  long long chunk = 0, c_end = 0;
  for (;;) {
    if (chunk >= c_end) {
      __syncthreads();  // every thread has read the previous s_grab
      if (threadIdx.x == 0) {
        const long long seen = (long long)*(volatile unsigned*)&b.ctl->chunk_next;  // a lower bound
        long long g = (nchunks - seen) / (2 * (long long)gridDim.x);
        g = g < 1 ? 1 : (g > BT_GRAB_MAX ? BT_GRAB_MAX : g);
        s_grab = (long long)atomicAdd(&b.ctl->chunk_next, (unsigned)g);
        s_len = g;
      }
      __syncthreads();
      chunk = s_grab;
      c_end = chunk + s_len < nchunks ? chunk + s_len : nchunks;
      if (chunk >= nchunks) break;
    }
    const long long base = chunk * BT_CHUNK;
    float v[BT_PER_THREAD][5];
    // per particle: -2 none, >= 0 local slot, <= -3 global slot -3 - ls (local table full); the
    // cell key is read back from the table, and the target found again from t0, so that no
    // per-particle key or target stays live across the barrier (the kernel runs at 64 registers)
    int ls[BT_PER_THREAD];
    const long long i0 = base + (long long)BT_PER_THREAD * threadIdx.x;
    const int t0 = i0 < N ? target_of(offs, b.T, i0) : 0;
    int t = t0;
    const float h0 = b.tg[t0].hf;  // the four particles' target is nearly always t0: its parameters once
    // the four consecutive particles of this thread with 16-byte loads and stores.  Row c of the
    // state and noise starts (c N) mod 4 floats off a 16-byte boundary: the thread reads the two
    // aligned quads around its four values (the second is the next thread's first, an L1 hit) and
    // shifts.  i0 + 8 <= N keeps the second quad of the last row inside the arrays.
    const bool vec = i0 + 8 <= N &&
                     ((reinterpret_cast<uintptr_t>(st) | reinterpret_cast<uintptr_t>(nz)) & 15u) == 0u;
    if (vec) {
      float4 sv[5], nv[5];
      if (DEF) {
        // deferred resampling: the four inputs gathered through the previous step's ancestors
        // (nondecreasing within a target, so a warp's reads stay within a few lines per row)
        const int4 a4 = *reinterpret_cast<const int4*>(b.ganc + i0);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const float* row = b.gsrc + c * P;
          sv[c] = make_float4(row[a4.x], row[a4.y], row[a4.z], row[a4.w]);
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const int m = (int)((c * N) & 3);
          const long long a = c * N + i0 - m;
          const float4 n0 = *reinterpret_cast<const float4*>(nz + a);
          nv[c] = m == 0 ? n0 : shift_quad(n0, *reinterpret_cast<const float4*>(nz + a + 4), m);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const int m = (int)((c * N) & 3);
          const long long a = c * N + i0 - m;
          const float4 s0 = *reinterpret_cast<const float4*>(st + a);
          const float4 n0 = *reinterpret_cast<const float4*>(nz + a);
          if (m == 0) {
            sv[c] = s0;
            nv[c] = n0;
          } else {
            sv[c] = shift_quad(s0, *reinterpret_cast<const float4*>(st + a + 4), m);
            nv[c] = shift_quad(n0, *reinterpret_cast<const float4*>(nz + a + 4), m);
          }
        }
      }
      const float* sp[5] = {&sv[0].x, &sv[1].x, &sv[2].x, &sv[3].x, &sv[4].x};
      const float* np[5] = {&nv[0].x, &nv[1].x, &nv[2].x, &nv[3].x, &nv[4].x};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[k][0] = __fadd_rn(__fadd_rn(sp[0][k], sp[2][k]), np[0][k]);
        v[k][1] = __fadd_rn(__fadd_rn(sp[1][k], sp[3][k]), np[1][k]);
        v[k][2] = __fadd_rn(sp[2][k], np[2][k]);
        v[k][3] = __fadd_rn(sp[3][k], np[3][k]);
        v[k][4] = __fadd_rn(sp[4][k], np[4][k]);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c)
        *reinterpret_cast<float4*>(b.prop + c * P + i0) = make_float4(v[0][c], v[1][c], v[2][c], v[3][c]);
    }
#pragma unroll
    for (int k = 0; k < BT_PER_THREAD; ++k) {
      const long long i = i0 + k;
      ls[k] = -2;
      if (i >= N) continue;
      while (t + 1 < b.T && offs[t + 1] <= i) ++t;
      if (!vec) {
        const float* sr = st;  // row c of the input state at sr + c rs
        long long rs = N, j = i;
        if (DEF) {
          sr = b.gsrc;
          rs = P;
          j = b.ganc[i];
        }
        const float x = sr[j], y = sr[rs + j], vx = sr[2 * rs + j], vy = sr[3 * rs + j], a = sr[4 * rs + j];
        v[k][0] = __fadd_rn(__fadd_rn(x, vx), nz[i]);
        v[k][1] = __fadd_rn(__fadd_rn(y, vy), nz[N + i]);
        v[k][2] = __fadd_rn(vx, nz[2 * N + i]);
        v[k][3] = __fadd_rn(vy, nz[3 * N + i]);
        v[k][4] = __fadd_rn(a, nz[4 * N + i]);
#pragma unroll
        for (int c = 0; c < 5; ++c) b.prop[c * P + i] = v[k][c];
      }
      const float h = t == t0 ? h0 : b.tg[t].hf;
      float fx = floorf(__fdiv_rn(__fadd_rn(v[k][0], 0.5f), h));
      float fy = floorf(__fdiv_rn(__fadd_rn(v[k][1], 0.5f), h));
      bool ok = fabsf(fx) < 33554431.0f && fabsf(fy) < 33554431.0f;
#pragma unroll
      for (int c = 0; c < 5; ++c) ok &= fabsf(v[k][c]) < 1.0e9f;
      if (!ok) {
        atomicOr(&b.ctl->err, (unsigned)PCSIR_DERR_RANGE);
        fx = fy = 0.0f;
        v[k][0] = v[k][1] = 0.0f;
      }
      const unsigned long long key = bkey(t, (int)fx, (int)fy);
      bool created;
      ls[k] = blocal_insert(tab, key, created);
      if (ls[k] == -1) ls[k] = -3 - (int)bglobal_insert(b, key);
    }
    __syncthreads();
    // global slots of the cells new in this chunk (list entries n_done .. n1): thread j claims entry
    // n_done + j, whose first compare-and-swap is issued here and completes while the thread sums
    // its particles below; the slots are read back after the chunk's closing barrier
    const unsigned n1 = tab.nlist;  // stable until the next chunk's insert pass
    const unsigned e_claim = n_done + threadIdx.x;
    unsigned long long claim_old = 0ull;
    if (e_claim < n1) {
      const unsigned long long ck = tab.key[tab.list[e_claim]];
      claim_old = atomicCAS(&b.hkey[hash_bits(ck, b.hbits)], EMPTY_KEY, ck);
    }
    // a thread's four particles are consecutive, and after resampling neighbours are often
    // offspring of one ancestor in one cell: a run of equal local slots is summed in registers
    // (exact integer pieces) and reaches the shared counters with one set of atomics
    unsigned run[BT_NACC];
#pragma unroll
    for (int a = 0; a < BT_NACC; ++a) run[a] = 0u;
    t = t0;
    const long long hq0 = b.tg[t0].hq;
    const long long an0 = b.st[t0].anchor[0], an1 = b.st[t0].anchor[1], an2 = b.st[t0].anchor[2];
#pragma unroll
    for (int k = 0; k < BT_PER_THREAD; ++k) {
      if (ls[k] == -2) continue;
      const long long i = i0 + k;
      while (t + 1 < b.T && offs[t + 1] <= i) ++t;
      const unsigned long long key = ls[k] >= 0 ? tab.key[ls[k]] : b.hkey[-3 - ls[k]];
      long long hq = hq0, a0 = an0, a1 = an1, a2 = an2;
      if (t != t0) {
        hq = b.tg[t].hq;
        a0 = b.st[t].anchor[0];
        a1 = b.st[t].anchor[1];
        a2 = b.st[t].anchor[2];
      }
      long long bv[5];
      bv[0] = to_fixed(v[k][0], 2147483648.0f) - (long long)bkey_bx(key) * hq + BT_POS_BIAS;
      bv[1] = to_fixed(v[k][1], 2147483648.0f) - (long long)bkey_by(key) * hq + BT_POS_BIAS;
      bv[2] = to_fixed(v[k][2], 4194304.0f) - a0 + BT_VAL_BIAS;
      bv[3] = to_fixed(v[k][3], 4194304.0f) - a1 + BT_VAL_BIAS;
      bv[4] = to_fixed(v[k][4], 4194304.0f) - a2 + BT_VAL_BIAS;
      bool bad = false;
#pragma unroll
      for (int c = 0; c < 5; ++c) bad |= (bv[c] < 0 || bv[c] >= BT_BIASED_LIMIT);
      if (bad) {
        atomicOr(&b.ctl->err, (unsigned)PCSIR_DERR_RANGE);
        bv[0] = bv[1] = BT_POS_BIAS;
        bv[2] = bv[3] = bv[4] = BT_VAL_BIAS;
      }
      if (ls[k] >= 0) {
        const int s = ls[k];
        run[0] += 1u;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          run[1 + 2 * c] += (unsigned)(bv[c] & BT_PIECE_MASK);
          run[2 + 2 * c] += (unsigned)(bv[c] >> BT_PIECE_BITS);
        }
        if (k == BT_PER_THREAD - 1 || ls[k + 1 < BT_PER_THREAD ? k + 1 : k] != s) {
          const unsigned old = atomicAdd(&tab.acc[0][s], run[0]);
          if (old < BT_HOT_AT && old + run[0] >= BT_HOT_AT) tab.hot = 1u;
          run[0] = 0u;
#pragma unroll
          for (int a = 1; a < BT_NACC; ++a) {
            atomicAdd(&tab.acc[a][s], run[a]);
            run[a] = 0u;
          }
        }
      } else {
        const unsigned g = (unsigned)(-3 - ls[k]);
        atomicAdd(&b.hcnt[g], 1u);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const long long bias = c < 2 ? BT_POS_BIAS : BT_VAL_BIAS;
          atomicAdd((unsigned long long*)&b.hsum[c * hcap + g], (unsigned long long)(bv[c] - bias));
        }
      }
    }
    {
      // the claims issued above: a slot that was empty is now this cell's (appended to the occupied
      // list, one append per warp), one that holds the key already was; on a collision the chain
      // continues from the next slot
      bool created = false;
      if (e_claim < n1) {
        const unsigned j = tab.list[e_claim];
        const unsigned long long ck = tab.key[j];
        const unsigned h0 = hash_bits(ck, b.hbits);
        unsigned g = h0;
        if (claim_old == EMPTY_KEY) created = true;
        else if (claim_old != ck) g = bglobal_claim(b, ck, created, (h0 + 1u) & ((1u << b.hbits) - 1u));
        tab.gslot[j] = g;
      }
      const unsigned lane = threadIdx.x & 31u;
      const unsigned m = __ballot_sync(0xffffffffu, created);
      if (m != 0u) {
        const unsigned leader = (unsigned)__ffs((int)m) - 1u;
        unsigned base = 0u;
        if (lane == leader) base = atomicAdd(&b.ctl->nocc, (unsigned)__popc((int)m));
        base = __shfl_sync(0xffffffffu, base, (int)leader);
        if (created)
          b.occ[base + (unsigned)__popc((int)(m & ((1u << lane) - 1u)))] = tab.gslot[tab.list[e_claim]];
      }
      if (n1 > n_done + blockDim.x) blocal_resolve(tab, b, n_done + blockDim.x, n1);  // more than one per thread
      n_new = n1 - n_done;
      n_done = n1;
      // the table is emptied after this chunk when it is full, or when a next chunk that met as many
      // new cells as this one would fill it: such a chunk (a block moving on to another target)
      // would otherwise send its particles past the full table to the global atomics one by one.
      // The fill is read here, between the two barriers, where no thread inserts (after the second
      // a thread may already insert the next chunk's cells), and the decision is read back after
      // the second (no thread writes it again before the next chunk's first).
      if (threadIdx.x == 0) s_clear = tab.fill + n_new >= BatchLocal<LTB>::CAP;
    }
    __syncthreads();
    // the slot of every particle: from the table for cells it holds (claimed above), from ls for the rest
    {
      unsigned gs[BT_PER_THREAD];
#pragma unroll
      for (int k = 0; k < BT_PER_THREAD; ++k)
        gs[k] = ls[k] >= 0 ? tab.gslot[ls[k]] : (unsigned)(-3 - ls[k]);
      if (vec) {
        *reinterpret_cast<uint4*>(b.pslot + i0) = make_uint4(gs[0], gs[1], gs[2], gs[3]);
      } else {
#pragma unroll
        for (int k = 0; k < BT_PER_THREAD; ++k)
          if (ls[k] != -2) b.pslot[i0 + k] = gs[k];
      }
    }
    // tab.hot is set only by the sums above and cleared below, both ordered by the barriers
    const bool full = s_clear;
    if (full || tab.hot != 0u) {
      blocal_flush(tab, b, full);
      if (full) n_done = 0u;
      // ordered before any count of the next chunk by that chunk's block barrier
      if (threadIdx.x == 0) tab.hot = 0u;
    }
    ++chunk;
  }
  blocal_flush(tab, b, false);
}

// ---------------------------------------------------------------------------
// Phase B: dummies and their likelihood, one warp per occupied cell
// ---------------------------------------------------------------------------
// The same with 32 / GS cells per warp (GS = 8 or 16 lanes each), for batches whose patches are
// all small (b.lik_group): the per-cell work (means, one-dimensional PSF factors, the group's sum)
// then runs for several cells at once instead of leaving most of a warp's lanes idle.
template <int GS>
__device__ void phase_bins_sub(const BatchBufs& b, const float* __restrict__ img, int W, int H, float* scratch_all) {
  constexpr int CPW = 32 / GS;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, grp = lane / GS, gtid = lane & (GS - 1);
  const unsigned B = *(volatile unsigned*)&b.ctl->nocc;
  const size_t hcap = size_t(1) << b.hbits;
  float* scratch = scratch_all + w * 4 * 64 + grp * (4 * 64 / CPW);
  const unsigned nw = gridDim.x * (blockDim.x >> 5);
  for (unsigned b0 = (blockIdx.x * (blockDim.x >> 5) + w) * CPW; b0 < B; b0 += nw * CPW) {
    const unsigned bi = b0 + grp;
    const bool active = bi < B;
    unsigned long long key = 0ull;
    int t = 0;
    unsigned n = 0u;
    LikParams lp{};
    LikPos pos{};
    if (active) {
      const unsigned g = b.occ[bi];
      key = b.hkey[g];
      t = bkey_t(key);
      const BatchTarget& T_ = b.tg[t];
      const BatchStats& S_ = b.st[t];
      n = b.hcnt[g];
      const double rdn = 1.0 / (double)n;  // one FP64 division per cell (GB300's FP64 rate is low)
      const double inv = 1.0 / 2147483648.0;
      const double mx = ((double)((long long)bkey_bx(key) * T_.hq) + (double)b.hsum[g] * rdn) * inv;
      const double my = ((double)((long long)bkey_by(key) * T_.hq) + (double)b.hsum[hcap + g] * rdn) * inv;
      const double mi = ((double)S_.anchor[2] + (double)b.hsum[4 * hcap + g] * rdn) * (1.0 / 4194304.0);
      lp.P = T_.patch;
      lp.kind = PCSIR_LIK_POISSON;
      lp.bg = T_.bg;
      lp.c2 = T_.c2;
      pos = lik_pos(mx, my, mi);
    }
    const LLSum ls = subgroup_loglik<GS>(img, W, H, pos, lp, scratch, active);
    const double ll = ll_to_double(ls);
    if (active && gtid == 0) {
      if (ls.bad) atomicOr(&b.ctl->err, (unsigned)PCSIR_DERR_NONFINITE);
      b.bin_ll[bi] = ll;
      b.bin_cnt[bi] = n;
      b.bin_key[bi] = key;
      if (!ls.bad) atomicMax(&b.st[t].max_ll, ord_encode(ll));
      atomicAdd(&b.st[t].nbins, 1u);
    }
  }
}

__device__ void phase_bins(const BatchBufs& b, const float* __restrict__ img, int W, int H, float* scratch_all) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned B = *(volatile unsigned*)&b.ctl->nocc;
  const size_t hcap = size_t(1) << b.hbits;
  float* scratch = scratch_all + w * 4 * 64;
  const unsigned nw = gridDim.x * (blockDim.x >> 5);
  for (unsigned bi = blockIdx.x * (blockDim.x >> 5) + w; bi < B; bi += nw) {
    const unsigned g = b.occ[bi];
    const unsigned long long key = b.hkey[g];
    const int t = bkey_t(key);
    const BatchTarget& T_ = b.tg[t];
    const BatchStats& S_ = b.st[t];
    const unsigned n = b.hcnt[g];
    const double dn = (double)n;
    const double rdn = 1.0 / dn;  // one FP64 division per cell (GB300's FP64 rate is low)
    const double inv = 1.0 / 2147483648.0;
    const double mx = ((double)((long long)bkey_bx(key) * T_.hq) + (double)b.hsum[g] * rdn) * inv;
    const double my = ((double)((long long)bkey_by(key) * T_.hq) + (double)b.hsum[hcap + g] * rdn) * inv;
    const double mi = ((double)S_.anchor[2] + (double)b.hsum[4 * hcap + g] * rdn) * (1.0 / 4194304.0);
    LikParams lp;
    lp.P = T_.patch;
    lp.kind = PCSIR_LIK_POISSON;
    lp.bg = T_.bg;
    lp.c2 = T_.c2;
    lp.inv2sxi2 = 0.0f;
    const LLSum ls = warp_loglik(img, W, H, lik_pos(mx, my, mi), lp, scratch);
    double ll = ll_to_double(ls);
    if (lane == 0) {
      if (ls.bad) atomicOr(&b.ctl->err, (unsigned)PCSIR_DERR_NONFINITE);
      b.bin_ll[bi] = ll;
      b.bin_cnt[bi] = n;
      b.bin_key[bi] = key;
      if (!ls.bad) atomicMax(&b.st[t].max_ll, ord_encode(ll));
      atomicAdd(&b.st[t].nbins, 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// Phase C: per-target weights of the cells, integer weights, sums
// ---------------------------------------------------------------------------
__device__ void phase_weights(const BatchBufs& b) {
  const unsigned B = *(volatile unsigned*)&b.ctl->nocc;
  const size_t hcap = size_t(1) << b.hbits;
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned bi = blockIdx.x * blockDim.x + threadIdx.x; bi < B; bi += stride) {
    const unsigned g = b.occ[bi];
    const unsigned long long key = b.hkey[g];
    const int t = bkey_t(key);
    BatchStats& S_ = b.st[t];
    const double m = ord_decode(*(volatile unsigned long long*)&S_.max_ll);
    const double ll = b.bin_ll[bi];
    const double wt = (ll == -INFINITY) ? 0.0 : exp(ll - m);
    const long long q = __double2ll_rn(ldexp(wt, b.tg[t].sq));
    b.hq[g] = q;
    const unsigned n = b.bin_cnt[bi];
    atomicAdd(&S_.T_f, n * wt);
    atomicAdd(&S_.T2_f, n * wt * wt);
    atomicAdd((unsigned long long*)&S_.T_int, (unsigned long long)((long long)n * q));
    const double inv = 1.0 / 2147483648.0;
    const double sx = (double)((long long)bkey_bx(key) * b.tg[t].hq) * inv * n + (double)b.hsum[g] * inv;
    const double sy = (double)((long long)bkey_by(key) * b.tg[t].hq) * inv * n + (double)b.hsum[hcap + g] * inv;
    atomicAdd(&S_.est[0], wt * sx);
    atomicAdd(&S_.est[1], wt * sy);
#pragma unroll
    for (int c = 2; c < 5; ++c) {
      const double sc = ((double)S_.anchor[c - 2] * n + (double)b.hsum[c * hcap + g]) * (1.0 / 4194304.0);
      atomicAdd(&S_.est[c], wt * sc);
    }
  }
}

// ---------------------------------------------------------------------------
// Phases D-F: resampling per (target, tile) item
// ---------------------------------------------------------------------------
__device__ __forceinline__ int item_target(const BatchBufs& b, int item) { return b.tile_target[item]; }

__device__ __forceinline__ long long bu_int(unsigned long long dhi, unsigned long long dlo, unsigned long long uhi,
                                            unsigned long long ulo, long long i) {
  const unsigned long long ui = (unsigned long long)i;
  const unsigned long long plo = ui * dlo;
  const unsigned long long phi = __umul64hi(ui, dlo);
  const unsigned long long s = plo + ulo;
  return (long long)(ui * dhi + uhi + phi + (s < plo ? 1ull : 0ull));
}

// first output i with U_i >= C (N if none; U_i = U0 + i Delta in 64.64 fixed point): a float
// guess of (C - U0) / Delta, then the exact integer correction
__device__ long long bfirst_out_f(const BatchStats& S, long long C, long long N) {
  if (C <= 0) return 0;
  if (S.dhi == 0ull && S.dlo == 0ull) return N;
  long long back;
  const float cf = i64_trunc_float(C - (long long)S.uhi, &back);
  const float xf = __fmul_rn(cf, S.inv_delta);
  long long i = xf <= 0.0f ? 0 : (xf >= (float)N ? N : (long long)__float2int_rn(xf));
  int guard = 0;
  while (i > 0 && bu_int(S.dhi, S.dlo, S.uhi, S.ulo, i - 1) >= C && guard++ < 256) --i;
  while (i < N && bu_int(S.dhi, S.dlo, S.uhi, S.ulo, i) < C && guard++ < 512) ++i;
  return i;
}

// number of the tile's cumulative weights C_j <= u, j < BT_TILE, over Cs padded as j + j / 16:
// while the search adds steps >= 16 the position stays a multiple of 16, so every probe is the
// running padded position plus a constant (the smaller steps never cross a pad)
__device__ __forceinline__ int btile_search(const long long* __restrict__ Cs, long long u) {
  int pa = 0;
#pragma unroll
  for (int step = BT_TILE / 2; step > 0; step >>= 1)
    if (Cs[pa + (step - 1) + ((step - 1) >> 4)] <= u) pa += step + (step >> 4);
  return pa - pa / 17;  // pa = 17 (a / 16) + a % 16
}

__device__ void phase_tile_sums(const BatchBufs& b) {
  __shared__ long long red[BT_THREADS / 32];
  for (int item = blockIdx.x; item < b.ntiles_total; item += gridDim.x) {
    const int t = item_target(b, item);
    const BatchTarget& T_ = b.tg[t];
    const long long base = T_.off + (long long)(item - T_.tile0) * BT_TILE;
    const long long end = T_.off + T_.n;
    long long s = 0;
    for (int j = threadIdx.x; j < BT_TILE; j += blockDim.x) {
      const long long i = base + j;
      if (i < end) s += b.hq[b.pslot[i]];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long tot = 0;
      for (int k = 0; k < BT_THREADS / 32; ++k) tot += red[k];
      b.tile_sum[item] = tot;
    }
    __syncthreads();
  }
}

// one thread per target: scan of its tile sums, the resampling map, the results
// one warp per target: the exclusive scan of the target's tile sums runs 32 tiles at a time
__device__ void phase_target_scan(const BatchBufs& b, const double* __restrict__ u0s) {
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < b.T; t += nwarps) {
    const BatchTarget& T_ = b.tg[t];
    BatchStats& S_ = b.st[t];
    long long e = 0;  // running total before the current group of 32 tiles
    for (int k0 = 0; k0 < T_.ntiles; k0 += 32) {
      const int k = k0 + lane;
      const long long v = k < T_.ntiles ? *(volatile long long*)&b.tile_sum[T_.tile0 + k] : 0ll;
      long long inc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
      }
      if (k < T_.ntiles) b.tile_excl[T_.tile0 + k] = e + inc - v;
      e += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane != 0) continue;
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
    pcsir_result& r = b.res[t];
    const double Tf = S_.T_f;
    for (int c = 0; c < 5; ++c) r.estimate[c] = S_.est[c] / Tf;
    r.ess = Tf * Tf / S_.T2_f;
    r.max_loglik = ord_decode(S_.max_ll);
    r.sum_wtilde = Tf;
    r.n_particles = T_.n;
    r.n_bins = S_.nbins;
    r.kind = 1;
    r.resampled = 1;
    r.device_error = Tq == 0ull ? PCSIR_DERR_ZEROSUM : 0;
  }
}

template <bool DEF>
__device__ void phase_resample(const BatchBufs& b, float* __restrict__ out, BatchResampleSmem& sm) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long Ntot = b.ntot;
  for (int item = blockIdx.x; item < b.ntiles_total; item += gridDim.x) {
    const int t = item_target(b, item);
    const BatchTarget& T_ = b.tg[t];
    const BatchStats& S_ = b.st[t];
    const long long lbase = (long long)(item - T_.tile0) * BT_TILE;  // within the target
    const long long N = T_.n;
    const int cnt = (int)((N - lbase) < BT_TILE ? (N - lbase) : BT_TILE);
    const long long excl = b.tile_excl[item];
    long long loc[BT_ITEMS];
    long long run = 0;
#pragma unroll
    for (int k = 0; k < BT_ITEMS; ++k) {
      const int j = tid * BT_ITEMS + k;
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
    if (lane == 31) sm.wtot[w] = inc;
    __syncthreads();
    long long woff = 0, agg = 0;
#pragma unroll
    for (int j = 0; j < BT_THREADS / 32; ++j) {
      const long long v = sm.wtot[j];
      if (j < w) woff += v;
      agg += v;
    }
    const long long texcl = woff + inc - run;
    // entries past the tile's last particle compare above every U_i (the fixed-step search below)
#pragma unroll
    for (int k = 0; k < BT_ITEMS; ++k) {
      const int jj = tid * BT_ITEMS + k;
      sm.Cs[jj + (jj >> 4)] = jj < cnt ? excl + texcl + loc[k] : LLONG_MAX;
    }
    // outputs [lo, hi) of the tile: U_lo >= C_{-1} = excl, U_{hi-1} < C_{cnt-1} = excl + agg
    if (tid == 0) sm.s_lo = bfirst_out_f(S_, excl, N);
    if (tid == 32) sm.s_hi = (lbase + cnt >= N) ? N : bfirst_out_f(S_, excl + agg, N);
    __syncthreads();
    const long long lo = sm.s_lo, hi = sm.s_hi;
    const bool zero_sum = (S_.dhi == 0ull && S_.dlo == 0ull);
    // four outputs per thread and pass.  Output i's ancestor is the tile's particle j with
    // C_{j-1} <= U_i < C_j, i.e. the number of C_j <= floor(U_i) (the C_j are integers): a
    // 12-step search over the cumulative weights in shared memory, independent for every
    // output, so a particle with many offspring does not serialise its thread
    for (long long i0 = lo + tid; i0 < hi; i0 += 4 * BT_THREADS) {
      long long src[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long long i = i0 + (long long)j * BT_THREADS;
        int a = 0;
        if (i < hi && !zero_sum) {
          a = btile_search(sm.Cs, bu_int(S_.dhi, S_.dlo, S_.uhi, S_.ulo, i));
          a = a < cnt ? a : cnt - 1;
        }
        // all weights zero: no distribution to sample, keep every particle
        src[j] = zero_sum ? T_.off + i : T_.off + lbase + a;
        if (b.anc != nullptr && i < hi) b.anc[T_.off + i] = (int)(src[j] - T_.off);
        if (DEF && i < hi) b.ganc[T_.off + i] = (int)src[j];
      }
      if (!DEF) {  // deferred: the next step gathers the states
        float v[4][5];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool has = i0 + (long long)j * BT_THREADS < hi;
#pragma unroll
          for (int d = 0; d < 5; ++d) v[j][d] = has ? b.prop[d * b.pstride + src[j]] : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const long long i = i0 + (long long)j * BT_THREADS;
          if (i < hi) {
#pragma unroll
            for (int d = 0; d < 5; ++d) out[d * Ntot + T_.off + i] = v[j][d];
          }
        }
      }
    }
    __syncthreads();
  }
}

template <int LTB, bool DEF>
__global__ void __launch_bounds__(BT_THREADS, 2)
k_batched_step(BatchBufs b, const float* __restrict__ st, const float* __restrict__ nz, float* __restrict__ out,
               const float* __restrict__ img, int W, int H, const double* __restrict__ u0s) {
  extern __shared__ __align__(16) unsigned char bt_smem[];
  long long* offs = reinterpret_cast<long long*>(bt_smem + bt_smem_union<LTB>());
  stamp(b.ctl, 0);
  // a step whose barrier wait ran out may have left cells in the table: clear all of it first
  // (ordered before every table access by the first barrier, after which block 0 lifts the mark)
  const bool was_dirty = *(volatile unsigned*)b.dirty != 0u;
  if (was_dirty) {
    const size_t hcap = size_t(1) << b.hbits;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < hcap; g += (size_t)gridDim.x * blockDim.x) {
      b.hkey[g] = EMPTY_KEY;
      b.hcnt[g] = 0u;
#pragma unroll
      for (int d = 0; d < 5; ++d) b.hsum[d * hcap + g] = 0;
    }
  }
  for (int t = threadIdx.x; t <= b.T; t += blockDim.x) offs[t] = b.offs[t];
  // anchors of vx, vy, I0 per target: the target's first particle's input value
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < b.T; t += gridDim.x * blockDim.x) {
    const long long i = b.tg[t].off;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float x = DEF ? b.gsrc[(2 + c) * b.pstride + b.ganc[i]] : st[(2 + c) * b.ntot + i];
      b.st[t].anchor[c] = to_fixed(x, 4194304.0f);
    }
  }
  if (!grid_barrier(b, 0)) return;
  if (was_dirty && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(b.dirty, 0u);
  stamp(b.ctl, 1);
  phase_prop_bin<LTB, DEF>(b, st, nz, *reinterpret_cast<BatchLocal<LTB>*>(bt_smem), offs);
  if (!grid_barrier(b, 1)) return;
  stamp(b.ctl, 2);
  if (b.lik_group == 8)
    phase_bins_sub<8>(b, img, W, H, reinterpret_cast<float*>(bt_smem));
  else if (b.lik_group == 16)
    phase_bins_sub<16>(b, img, W, H, reinterpret_cast<float*>(bt_smem));
  else
    phase_bins(b, img, W, H, reinterpret_cast<float*>(bt_smem));
  if (!grid_barrier(b, 2)) return;
  stamp(b.ctl, 3);
  phase_weights(b);
  // the cells are not needed any more: return their hash slots to empty
  // after the tile sums, which still read the slots' integer weights
  if (!grid_barrier(b, 3)) return;
  stamp(b.ctl, 4);
  phase_tile_sums(b);
  if (!grid_barrier(b, 4)) return;
  stamp(b.ctl, 5);
  phase_target_scan(b, u0s);
  {
    const unsigned B = *(volatile unsigned*)&b.ctl->nocc;
    const size_t hcap = size_t(1) << b.hbits;
    for (unsigned bi = blockIdx.x * blockDim.x + threadIdx.x; bi < B; bi += gridDim.x * blockDim.x) {
      const unsigned g = b.occ[bi];
      b.hkey[g] = EMPTY_KEY;
      b.hcnt[g] = 0u;
#pragma unroll
      for (int d = 0; d < 5; ++d) b.hsum[d * hcap + g] = 0;
    }
  }
  if (!grid_barrier(b, 5)) return;
  stamp(b.ctl, 6);
  phase_resample<DEF>(b, out, *reinterpret_cast<BatchResampleSmem*>(bt_smem));
  if (!grid_barrier(b, 6)) return;
  stamp(b.ctl, 7);
}

// the kernel variant of a cell-table size and its dynamic shared memory
const void* bt_kernel(int ltb, bool def = false) {
  switch (ltb) {
    case 9: return def ? reinterpret_cast<const void*>(k_batched_step<9, true>)
                       : reinterpret_cast<const void*>(k_batched_step<9, false>);
    case 11: return def ? reinterpret_cast<const void*>(k_batched_step<11, true>)
                        : reinterpret_cast<const void*>(k_batched_step<11, false>);
    default: return def ? reinterpret_cast<const void*>(k_batched_step<10, true>)
                        : reinterpret_cast<const void*>(k_batched_step<10, false>);
  }
}
size_t bt_smem_bytes(int ltb) {
  return ltb == 9 ? bt_smem<9>() : (ltb == 11 ? bt_smem<11>() : bt_smem<10>());
}
// blocks per SM that fit, for both variants of the kernel (plain and deferred resampling)
cudaError_t bt_blocks_per_sm(int ltb, int* per_sm) {
  int a = 0, d = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, bt_kernel(ltb, false), BT_THREADS,
                                                                bt_smem_bytes(ltb));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, bt_kernel(ltb, true), BT_THREADS, bt_smem_bytes(ltb));
  *per_sm = a < d ? a : d;
  return e;
}

}  // namespace pcsir

// ---------------------------------------------------------------------------
// Host API
// ---------------------------------------------------------------------------
using namespace pcsir;

struct pcsir_batch {
  int T = 0;
  long long ntot = 0;
  int ntiles = 0;
  int grid = 0;
  int ltb = BT_LTB_DEFAULT;  // cell-table bits of the kernel variant
  BatchBufs b{};
  std::vector<void*> allocs;
  pcsir_result* host_res = nullptr;
  std::string err = "no error";
  bool failed = false;
  // deferred resampling: b.prop alternates between the two state buffers (the step gathers from
  // the one the previous step wrote and writes the other); def_anc holds the last resampling's
  // ancestors as global indices
  float* prop_main = nullptr;
  float* prop_alt = nullptr;
  int* def_anc = nullptr;
  bool def_active = false;
};

namespace {
template <typename X>
bool balloc(pcsir_batch* c, X** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(X) + 16) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->allocs.push_back(q);
  *p = static_cast<X*>(q);
  return true;
}
void bfree(pcsir_batch* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->host_res) cudaFreeHost(c->host_res);
  c->host_res = nullptr;
}
}  // namespace

extern "C" {

pcsir_status pcsir_batch_create(const pcsir_target* targets, int32_t T, pcsir_batch** out) {
  if (!out) return PCSIR_EINVAL;
  *out = nullptr;
  if (!targets || T < 1 || T > BT_MAX_TARGETS) return PCSIR_EINVAL;
  long long ntot = 0;
  int ntiles = 0;
  std::vector<BatchTarget> tg(T);
  for (int t = 0; t < T; ++t) {
    const pcsir_target& x = targets[t];
    if (x.n_particles < 1 || !(x.h > 0.0 && x.h <= MAX_H) || !(x.psf_sigma > 0.0) || !(x.bg > 0.0) ||
        x.patch < 1 || x.patch > 63 || (x.patch & 1) == 0)
      return PCSIR_EINVAL;
    tg[t].off = ntot;
    tg[t].n = x.n_particles;
    tg[t].h = (double)(float)x.h;
    tg[t].hf = (float)x.h;
    {
      const double c2 = 1.0 / (2.0 * x.psf_sigma * x.psf_sigma);
      tg[t].c2.hi = (float)c2;
      tg[t].c2.lo = (float)(c2 - (double)tg[t].c2.hi);
    }
    tg[t].hq = llrint(x.h * 2147483648.0);
    tg[t].sigma = x.psf_sigma;
    tg[t].bg = (float)x.bg;
    tg[t].patch = x.patch;
    tg[t].sq = weight_scale_bits(x.n_particles);
    tg[t].tile0 = ntiles;
    tg[t].ntiles = (int)((x.n_particles + BT_TILE - 1) / BT_TILE);

    ntot += x.n_particles;
    ntiles += tg[t].ntiles;
  }
  if (ntot > MAX_PARTICLES) return PCSIR_ERANGE;
  pcsir_batch* c = new (std::nothrow) pcsir_batch();
  if (!c) return PCSIR_ENOMEM;
  c->T = T;
  c->ntot = ntot;
  c->ntiles = ntiles;
  int hbits = 10;
  while ((1ll << hbits) < 2 * ntot) ++hbits;
  const size_t hcap = size_t(1) << hbits;
  BatchBufs& b = c->b;
  b.T = T;
  b.ntot = ntot;
  b.pstride = (ntot + 3) & ~3ll;
  b.ntiles_total = ntiles;
  b.hbits = hbits;
  {
    int pmax = 0;
    for (int t = 0; t < T; ++t) pmax = std::max(pmax, tg[t].patch);
    b.lik_group = pmax <= 15 ? 8 : (pmax <= 31 ? 16 : 32);
  }
  BatchTarget* dtg = nullptr;
  long long* doffs = nullptr;
  int* dtile_target = nullptr;
  bool ok = balloc(c, &dtg, T) && balloc(c, &b.st, T) && balloc(c, &b.ctl, 1) && balloc(c, &doffs, T + 1) &&
            balloc(c, &b.hkey, hcap) && balloc(c, &b.hcnt, hcap) && balloc(c, &b.hsum, 5 * hcap) &&
            balloc(c, &b.hq, hcap) && balloc(c, &b.occ, (size_t)ntot) && balloc(c, &b.bin_ll, (size_t)ntot) &&
            balloc(c, &b.bin_cnt, (size_t)ntot) && balloc(c, &b.bin_key, (size_t)ntot) &&
            balloc(c, &b.pslot, (size_t)ntot) &&
            balloc(c, &b.prop, 5 * (size_t)b.pstride) && balloc(c, &b.tile_sum, (size_t)ntiles) &&
            balloc(c, &b.tile_excl, (size_t)ntiles) && balloc(c, &b.res, (size_t)T) &&
            balloc(c, &dtile_target, (size_t)ntiles) && balloc(c, &b.dirty, 1);
  if (!ok) {
    bfree(c);
    delete c;
    return PCSIR_ENOMEM;
  }
  b.tg = dtg;
  b.offs = doffs;
  c->prop_main = b.prop;
  b.gsrc = nullptr;
  b.ganc = nullptr;
  b.tile_target = dtile_target;
  b.anc = nullptr;
  b.qout = nullptr;
  b.bar_spins = BT_BARRIER_SPINS;
  b.bar_fail = -1;
  std::vector<long long> offs(T + 1);
  for (int t = 0; t < T; ++t) offs[t] = tg[t].off;
  offs[T] = ntot;
  std::vector<int> tile_target(ntiles);
  for (int t = 0; t < T; ++t)
    for (int k = 0; k < tg[t].ntiles; ++k) tile_target[tg[t].tile0 + k] = t;
  cudaError_t e = cudaMemcpy(dtg, tg.data(), sizeof(BatchTarget) * T, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(dtile_target, tile_target.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(doffs, offs.data(), sizeof(long long) * (T + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b.hkey, 0xff, hcap * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(b.hcnt, 0, hcap * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(b.hsum, 0, 5 * hcap * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(b.dirty, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMallocHost(&c->host_res, sizeof(pcsir_result) * T);
  for (int ltb = BT_LTB_MIN; ltb <= BT_LTB_MAX && e == cudaSuccess; ++ltb)
    for (int def = 0; def < 2 && e == cudaSuccess; ++def)
      e = cudaFuncSetAttribute(bt_kernel(ltb, def != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)bt_smem_bytes(ltb));
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess) e = bt_blocks_per_sm(BT_LTB_DEFAULT, &per_sm);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess || !coop || per_sm < 1) {
    cudaGetLastError();
    bfree(c);
    delete c;
    return e == cudaErrorMemoryAllocation ? PCSIR_ENOMEM : (e != cudaSuccess ? PCSIR_ECUDA : PCSIR_ENOTSUP);
  }
  c->grid = sms * per_sm;
  *out = c;
  return PCSIR_OK;
}

pcsir_status pcsir_batch_set_grid(pcsir_batch* c, int32_t blocks_per_sm) {
  if (!c || blocks_per_sm < 1) return PCSIR_EINVAL;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = bt_blocks_per_sm(c->ltb, &per_sm);
  if (e != cudaSuccess) return PCSIR_ECUDA;
  if (blocks_per_sm > per_sm) return PCSIR_ERANGE;
  c->grid = sms * blocks_per_sm;
  return PCSIR_OK;
}

pcsir_status pcsir_batch_set_table(pcsir_batch* c, int32_t table_bits) {
  if (!c || table_bits < BT_LTB_MIN || table_bits > BT_LTB_MAX) return PCSIR_EINVAL;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = bt_blocks_per_sm(table_bits, &per_sm);
  if (e != cudaSuccess) return PCSIR_ECUDA;
  if (per_sm < 1) return PCSIR_ERANGE;
  c->ltb = table_bits;
  if (c->grid > sms * per_sm) c->grid = sms * per_sm;  // the larger table fits fewer blocks per SM
  return PCSIR_OK;
}

pcsir_status pcsir_batch_destroy(pcsir_batch* c) {
  if (!c) return PCSIR_OK;
  cudaDeviceSynchronize();
  bfree(c);
  delete c;
  return PCSIR_OK;
}

// the cooperative launch of one step and the copy of its results
static pcsir_status bt_launch(pcsir_batch* c, BatchBufs b, const float* st_in, const float* nz, float* out,
                              const float* img, int w, int h, const double* u0s, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b.ctl, 0, sizeof(BatchCtl), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.st, 0, sizeof(BatchStats) * c->T, s);
  if (e == cudaSuccess) {
    void* args[] = {&b, &st_in, &nz, &out, &img, &w, &h, &u0s};
    e = cudaLaunchCooperativeKernel(bt_kernel(c->ltb, b.gsrc != nullptr), dim3(c->grid), dim3(BT_THREADS), args, bt_smem_bytes(c->ltb),
                                    s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->host_res, b.res, sizeof(pcsir_result) * c->T, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) {
    c->err = std::string("batched step: ") + cudaGetErrorString(e);
    c->failed = true;
    return PCSIR_ECUDA;
  }
  return PCSIR_OK;
}

pcsir_status pcsir_batched_step(pcsir_batch* c, float* state, const float* image, int32_t W, int32_t H,
                                const float* noise, const double* u0, void* stream) {
  if (!c) return PCSIR_EINVAL;
  if (c->failed) return PCSIR_ESTATE;
  if (!state || !image || !noise || !u0 || W < 1 || H < 1) {
    c->err = "NULL pointer or empty image";
    return PCSIR_EINVAL;
  }
  c->def_active = false;  // a plain step ends a deferred run
  return bt_launch(c, c->b, state, noise, state, image, W, H, u0, static_cast<cudaStream_t>(stream));
}

__global__ void k_bt_iota(int* __restrict__ a, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] = (int)i;
}

// out[c][i] = src[c][anc[i]]: the resampled states of a deferred run, rows of n (out) and P (src) floats
__global__ void k_bt_gather(float* __restrict__ out, const float* __restrict__ src, long long P,
                            const int* __restrict__ anc, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long a = anc[i];
#pragma unroll
    for (int r = 0; r < 5; ++r) out[r * n + i] = src[r * P + a];
  }
}

static int bt_elem_grid(const pcsir_batch* c) {
  const long long g = (c->ntot + 255) / 256;
  return (int)std::min<long long>(g, (long long)c->grid * 8);
}

pcsir_status pcsir_batch_deferred_begin(pcsir_batch* c, const float* state, void* stream) {
  if (!c) return PCSIR_EINVAL;
  if (c->failed) return PCSIR_ESTATE;
  if (!state) {
    c->err = "NULL state";
    return PCSIR_EINVAL;
  }
  if ((!c->prop_alt && !balloc(c, &c->prop_alt, 5 * (size_t)c->b.pstride)) ||
      (!c->def_anc && !balloc(c, &c->def_anc, (size_t)c->ntot))) {
    c->err = "deferred run: out of device memory";
    return PCSIR_ENOMEM;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t row = sizeof(float) * (size_t)c->ntot;
  cudaError_t e = cudaMemcpy2DAsync(c->b.prop, sizeof(float) * (size_t)c->b.pstride, state, row, row, 5,
                                    cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) {
    k_bt_iota<<<bt_elem_grid(c), 256, 0, s>>>(c->def_anc, c->ntot);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    c->err = std::string("deferred begin: ") + cudaGetErrorString(e);
    c->failed = true;
    return PCSIR_ECUDA;
  }
  c->def_active = true;
  return PCSIR_OK;
}

pcsir_status pcsir_batched_deferred_step(pcsir_batch* c, const float* image, int32_t W, int32_t H, const float* noise,
                                         const double* u0, void* stream) {
  if (!c) return PCSIR_EINVAL;
  if (c->failed || !c->def_active) {
    if (!c->def_active) c->err = "no deferred run: call pcsir_batch_deferred_begin first";
    return PCSIR_ESTATE;
  }
  if (!image || !noise || !u0 || W < 1 || H < 1) {
    c->err = "NULL pointer or empty image";
    return PCSIR_EINVAL;
  }
  BatchBufs b = c->b;
  b.gsrc = c->b.prop;
  b.ganc = c->def_anc;
  b.prop = c->b.prop == c->prop_main ? c->prop_alt : c->prop_main;
  const pcsir_status st = bt_launch(c, b, nullptr, noise, nullptr, image, W, H, u0, static_cast<cudaStream_t>(stream));
  if (st == PCSIR_OK) c->b.prop = b.prop;
  return st;
}

pcsir_status pcsir_batch_deferred_state(pcsir_batch* c, float* state, void* stream) {
  if (!c) return PCSIR_EINVAL;
  if (c->failed || !c->def_active) {
    if (!c->def_active) c->err = "no deferred run: call pcsir_batch_deferred_begin first";
    return PCSIR_ESTATE;
  }
  if (!state) {
    c->err = "NULL state";
    return PCSIR_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_bt_gather<<<bt_elem_grid(c), 256, 0, s>>>(state, c->b.prop, c->b.pstride, c->def_anc, c->ntot);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->err = std::string("deferred state: ") + cudaGetErrorString(e);
    c->failed = true;
    return PCSIR_ECUDA;
  }
  return PCSIR_OK;
}

pcsir_status pcsir_batch_results(pcsir_batch* c, pcsir_result* out, int32_t T, int32_t* device_error) {
  if (!c || !out || T != c->T) return PCSIR_EINVAL;
  // the step's copy of the results to page-locked memory is asynchronous: wait for it
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return PCSIR_ECUDA;
  }
  std::memcpy(out, c->host_res, sizeof(pcsir_result) * T);
  if (device_error) {
    BatchCtl ctl;
    if (cudaMemcpy(&ctl, c->b.ctl, sizeof(ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return PCSIR_ECUDA;
    *device_error = (int32_t)ctl.err;
    if (ctl.err & PCSIR_DERR_TIMEOUT) return PCSIR_ETIMEDOUT;
  }
  return PCSIR_OK;
}

pcsir_status pcsir_batch_set_wait(pcsir_batch* c, int32_t max_polls, int32_t unreachable_barrier) {
  if (!c || max_polls < 1 || unreachable_barrier < -1 || unreachable_barrier >= BT_NBARRIERS) return PCSIR_EINVAL;
  c->b.bar_spins = max_polls;
  c->b.bar_fail = unreachable_barrier;
  return PCSIR_OK;
}

pcsir_status pcsir_batch_keep(pcsir_batch* c, int32_t keep) {
  if (!c || (keep & ~(PCSIR_KEEP_ANCESTORS | PCSIR_KEEP_QWEIGHTS))) return PCSIR_EINVAL;
  if (c->failed) return PCSIR_ESTATE;
  bool ok = true;
  if ((keep & PCSIR_KEEP_ANCESTORS) && !c->b.anc) ok = balloc(c, &c->b.anc, (size_t)c->ntot);
  if (ok && (keep & PCSIR_KEEP_QWEIGHTS) && !c->b.qout) ok = balloc(c, &c->b.qout, (size_t)c->ntot);
  return ok ? PCSIR_OK : PCSIR_ENOMEM;
}

pcsir_status pcsir_batch_kept(pcsir_batch* c, const int32_t** ancestor, const int64_t** qweight) {
  if (!c) return PCSIR_EINVAL;
  if (ancestor) *ancestor = c->b.anc;
  if (qweight) *qweight = reinterpret_cast<const int64_t*>(c->b.qout);
  return PCSIR_OK;
}

pcsir_status pcsir_batch_outputs(pcsir_batch* c, const float** prop_state, int64_t* row_stride,
                                 const unsigned int** particle_slot, int64_t* n_total) {
  if (!c) return PCSIR_EINVAL;
  if (prop_state) *prop_state = c->b.prop;
  if (row_stride) *row_stride = c->b.pstride;
  if (particle_slot) *particle_slot = c->b.pslot;
  if (n_total) *n_total = c->ntot;
  return PCSIR_OK;
}

pcsir_status pcsir_batch_bins(pcsir_batch* c, const uint64_t** keys, const uint32_t** counts, const double** loglik,
                              int64_t* n_bins) {
  if (!c) return PCSIR_EINVAL;
  if (keys) *keys = reinterpret_cast<const uint64_t*>(c->b.bin_key);
  if (counts) *counts = c->b.bin_cnt;
  if (loglik) *loglik = c->b.bin_ll;
  if (n_bins) {
    BatchCtl ctl;
    if (cudaMemcpy(&ctl, c->b.ctl, sizeof(ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return PCSIR_ECUDA;
    *n_bins = ctl.nocc;
  }
  return PCSIR_OK;
}

const char* pcsir_batch_last_error(pcsir_batch* c) { return c ? c->err.c_str() : "NULL batch"; }

pcsir_status pcsir_batch_phase_times(pcsir_batch* c, double* ms, int32_t n) {
  if (!c || !ms || n < 7) return PCSIR_EINVAL;
  BatchCtl h{};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, c->b.ctl, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PCSIR_ECUDA;
  }
  for (int k = 0; k < 7; ++k) ms[k] = (double)(h.phase_ns[k + 1] - h.phase_ns[k]) * 1e-6;
  return PCSIR_OK;
}

}  // extern "C"
