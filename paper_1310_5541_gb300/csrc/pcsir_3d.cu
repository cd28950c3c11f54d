// pcSIR and SIR for 3D tracking (include/pcsir3.h): state (x, y, z, vx, vy,
// vz, I0) in float32 structure-of-arrays, 3D cells over position, dummies at
// the cells' centres of mass, the Poisson likelihood of an anisotropic
// Gaussian PSF over a patch_xy x patch_xy x patch_z voxel block, and the
// systematic resampling of pcsir_resample.cu (instantiated for seven
// components).
//
// The propagate/cell kernel follows the 2D one: a block-private hash table
// of cells in shared memory with exact fixed-point sums (count and two
// 18-bit pieces per biased component, 32-bit shared atomics), flushed to a
// global open-addressing table with 64-bit integer atomics.  Positions are
// offsets from the cell origin at 2^-31 voxel, the other four components
// offsets from particle 0's input value at 2^-22.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pcsir_3d.cuh"
#include "pcsir_surrogate.h"

namespace pcsir {

struct Step3 {
  StepBuffers b;      // hsum [7][hcap], dummy [7][stride], prop [7][N]
  int32_t* bin_xyz;   // [3][stride]
  pcsir3_result* dres3;
};

// ---------------------------------------------------------------------------
// Propagate + cell + centre-of-mass sums (Algorithm 2, 3D)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(P3_THREADS, 2)
k_prop_bin3(StepBuffers b, const float* __restrict__ st, const float* __restrict__ nz, int64_t N, float hx, float hy,
            float hz, long long hqx, long long hqy, long long hqz) {
  extern __shared__ __align__(16) unsigned char smem3[];
  Local3& tab = *reinterpret_cast<Local3*>(smem3);
  float* __restrict__ prop = static_cast<float*>(b.prop);
  const size_t hcap = size_t(1) << b.hbits;
  for (int j = threadIdx.x; j < L3; j += blockDim.x) {
    tab.key[j] = EMPTY_KEY;
#pragma unroll
    for (int a = 0; a < NACC3; ++a) tab.acc[a][j] = 0u;
  }
  if (threadIdx.x == 0) {
    tab.fill = 0u;
    tab.hot = 0u;
  }
  long long anc[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) anc[c] = to_fixed(st[(3 + c) * N], 4194304.0f);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) b.ctl->anchor[3 + c] = anc[c];
  }
  __syncthreads();
  const float lim = 1048575.0f;  // |cell index| < 2^20
  const float hh[3] = {hx, hy, hz};
  const long long hq[3] = {hqx, hqy, hqz};
  const int64_t nchunks = (N + P3_CHUNK - 1) / P3_CHUNK;
  for (int64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const int64_t base = chunk * P3_CHUNK;
    float v[P3_PER_THREAD][NS3];
    // each particle is summed into its cell as soon as the cell is found; ls: the cell's local
    // slot, -3 - its global slot (table full), or -2 (no particle)
    int ls[P3_PER_THREAD];
    bool flag = false;  // this thread filled the table or brought a cell's count to the flush mark
#pragma unroll
    for (int k = 0; k < P3_PER_THREAD; ++k) {
      const int64_t i = base + (int64_t)k * P3_THREADS + threadIdx.x;
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
      const int64_t i = base + (int64_t)k * P3_THREADS + threadIdx.x;
      if (i >= N) continue;
      bool ok = true;
      float f[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        f[p] = floorf(__fdiv_rn(__fadd_rn(v[k][p], 0.5f), hh[p]));
        ok &= fabsf(f[p]) < lim;
      }
#pragma unroll
      for (int c = 0; c < NS3; ++c) ok &= fabsf(v[k][c]) < 1.0e9f;
      if (!ok) {
        raise_flag(b.ctl, PCSIR_DERR_RANGE);
        f[0] = f[1] = f[2] = 0.0f;
        v[k][0] = v[k][1] = v[k][2] = 0.0f;
      }
      int bidx[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) bidx[p] = (int)f[p];
      const unsigned long long key = pack_key3(bidx[0], bidx[1], bidx[2]);
      bool created;
      int s = local_insert3(tab, key, created, flag);
      if (created) tab.gslot[s] = global_insert3(b, key);
      long long bv[NS3];
#pragma unroll
      for (int p = 0; p < 3; ++p) bv[p] = to_fixed(v[k][p], 2147483648.0f) - (long long)bidx[p] * hq[p] + P3_POS_BIAS;
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[3 + c] = to_fixed(v[k][3 + c], 4194304.0f) - anc[c] + P3_VAL_BIAS;
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
      const int64_t i = base + (int64_t)k * P3_THREADS + threadIdx.x;
      b.pslot[i] = ls[k] >= 0 ? tab.gslot[ls[k]] : (unsigned)(-3 - ls[k]);
    }
    if (flush) local_flush3(tab, b, tab.fill >= L3_CAP);  // read before the flush's first barrier
  }
  local_flush3(tab, b, false);
}

// ---------------------------------------------------------------------------
// Dummies and their likelihood: one warp per occupied cell
// ---------------------------------------------------------------------------
constexpr int B3_THREADS = 256;

__device__ __forceinline__ void block_max3(double v, Control* ctl) {
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

// 3D cells: the key packs (bx + 2^20, by + 2^20, bz + 2^20) in 21-bit fields
__device__ __forceinline__ bool sur_held3(int bx, int by, int bz, unsigned long long salt, unsigned thr) {
  const unsigned long long key = (unsigned long long)(unsigned)(bx + (1 << 20)) |
                                 ((unsigned long long)(unsigned)(by + (1 << 20)) << 21) |
                                 ((unsigned long long)(unsigned)(bz + (1 << 20)) << 42);
  const unsigned long long h = splitmix64(key + salt * 0x9E3779B97F4A7C15ull);
  return (unsigned)(h >> 40) < thr;
}

// held-out selection and list of a surrogate-assisted step (SUR)
struct SurBins3 {
  unsigned long long salt;
  double frac;
  int min_holdout;
  int ho_cap;
  int* ho_bin;
  double* ho_ll;
  SurStats* stats;
};

template <bool SUR>
__global__ void __launch_bounds__(B3_THREADS)
k_bins3(StepBuffers b, int32_t* __restrict__ bin_xyz, Lik3 lp, const float* __restrict__ vol, int W, int H, int D,
        long long hqx, long long hqy, long long hqz, SurBins3 sb) {
  constexpr int NW = B3_THREADS / 32;
  __shared__ float scratch[NW][2 * (3 * MAXP3)];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned B = b.ctl->nocc;
  const size_t hcap = size_t(1) << b.hbits;
  const int64_t bs = b.bin_stride;
  const long long hq[3] = {hqx, hqy, hqz};
  const unsigned thr = SUR ? sur_holdout_threshold(sb.frac, sb.min_holdout, B) : 0u;
  double mymax = -INFINITY;
  for (unsigned bi = blockIdx.x * NW + w; bi < B; bi += gridDim.x * NW) {
    const unsigned g = b.occ[bi];
    const unsigned long long key = b.hkey[g];
    const double dn = (double)b.hcnt[g];
    const double rdn = 1.0 / dn;  // one FP64 division per cell (GB300's FP64 rate is low)
    double mean[NS3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
      mean[p] = ((double)((long long)key3(key, p) * hq[p]) + (double)b.hsum[p * hcap + g] * rdn) * POS_INV;
#pragma unroll
    for (int c = 3; c < NS3; ++c) mean[c] = ((double)b.ctl->anchor[c] + (double)b.hsum[c * hcap + g] * rdn) * VAL_INV;
    if (lane == 0) {
#pragma unroll
      for (int p = 0; p < 3; ++p) bin_xyz[p * bs + bi] = key3(key, p);
      b.bin_cnt[bi] = b.hcnt[g];
#pragma unroll
      for (int c = 0; c < NS3; ++c) b.dummy[c * bs + bi] = mean[c];
      b.hrank[g] = bi;
    }
    bool held = false;
    if (SUR) {
      // the surrogate predicts every dummy whose 11 x 11 x 7 patch lies inside the volume,
      // except the held-out ones
      const int rxy = lp.Pxy >> 1, rz = lp.Pz >> 1;
      const double fx = floor(mean[0] + 0.5), fy = floor(mean[1] + 0.5), fz = floor(mean[2] + 0.5);
      const bool clipped = !(fx - rxy >= 0.0 && fx + rxy <= (double)(W - 1) && fy - rxy >= 0.0 &&
                             fy + rxy <= (double)(H - 1) && fz - rz >= 0.0 && fz + rz <= (double)(D - 1));
      held = !clipped && sur_held3(key3(key, 0), key3(key, 1), key3(key, 2), sb.salt, thr);
      if (!clipped && !held) continue;  // uniform over the warp
      if (!held && lane == 0) atomicAdd(&sb.stats->n_clipped, 1u);
    }
    double ll = ll_to_double(warp_loglik3(vol, W, H, D, pos3(mean[0], mean[1], mean[2], mean[6]), lp, scratch[w]));
    if (!isfinite(ll)) {
      if (lane == 0) raise_flag(b.ctl, PCSIR_DERR_NONFINITE);
      ll = -INFINITY;
    }
    if (SUR && held) {
      if (lane == 0) {
        const unsigned slot = atomicAdd(&sb.stats->n_ho, 1u);
        if (slot < (unsigned)sb.ho_cap) {
          sb.ho_bin[slot] = (int)bi;
          sb.ho_ll[slot] = ll;
        }
      }
      continue;
    }
    if (lane == 0) b.bin_ll[bi] = ll;
    mymax = fmax(mymax, ll);
  }
  block_max3(mymax, b.ctl);
}

// Exact likelihood of every dummy when the held-out check rejected the surrogate's
// predictions (stats->fallback); otherwise returns at once.  The dummies are those
// k_bins3 stored, so the values equal the plain step's.
__global__ void __launch_bounds__(B3_THREADS)
k_bins3_fallback(StepBuffers b, Lik3 lp, const float* __restrict__ vol, int W, int H, int D,
                 const SurStats* __restrict__ stats) {
  if (*(volatile const unsigned*)&stats->fallback == 0u) return;
  constexpr int NW = B3_THREADS / 32;
  __shared__ float scratch[NW][2 * (3 * MAXP3)];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned B = b.ctl->nocc;
  const int64_t bs = b.bin_stride;
  double mymax = -INFINITY;
  for (unsigned bi = blockIdx.x * NW + w; bi < B; bi += gridDim.x * NW) {
    const double x = b.dummy[bi], y = b.dummy[bs + bi], z = b.dummy[2 * bs + bi], a = b.dummy[6 * bs + bi];
    double ll = ll_to_double(warp_loglik3(vol, W, H, D, pos3(x, y, z, a), lp, scratch[w]));
    if (!isfinite(ll)) {
      if (lane == 0) raise_flag(b.ctl, PCSIR_DERR_NONFINITE);
      ll = -INFINITY;
    }
    if (lane == 0) b.bin_ll[bi] = ll;
    mymax = fmax(mymax, ll);
  }
  block_max3(mymax, b.ctl);
}

// ---------------------------------------------------------------------------
// Weight reductions and the step's results (7 components)
// ---------------------------------------------------------------------------
constexpr int R3_THREADS = 256;

struct Red3 {
  double Tf, T2, est[NS3];
  long long Tint;
};

__device__ void commit3(Red3 a, const StepBuffers& b, pcsir3_result* r, int64_t N, int kind, unsigned nblocks) {
  __shared__ double sd[2 + NS3][R3_THREADS / 32];
  __shared__ long long sl[R3_THREADS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double vals[2 + NS3];
  vals[0] = a.Tf;
  vals[1] = a.T2;
#pragma unroll
  for (int c = 0; c < NS3; ++c) vals[2 + c] = a.est[c];
  long long ti = a.Tint;
#pragma unroll
  for (int k = 0; k < 2 + NS3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vals[k] += __shfl_xor_sync(0xffffffffu, vals[k], o);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ti += __shfl_xor_sync(0xffffffffu, ti, o);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 2 + NS3; ++k) sd[k][w] = vals[k];
    sl[w] = ti;
  }
  __syncthreads();
  Control* ctl = b.ctl;
  if (threadIdx.x == 0) {
    double t[2 + NS3] = {};
    long long tt = 0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) {
#pragma unroll
      for (int k = 0; k < 2 + NS3; ++k) t[k] += sd[k][j];
      tt += sl[j];
    }
    atomicAdd(&ctl->T_f, t[0]);
    atomicAdd(&ctl->T2_f, t[1]);
#pragma unroll
    for (int c = 0; c < NS3; ++c) atomicAdd(&ctl->est[c], t[2 + c]);
    atomicAdd((unsigned long long*)&ctl->T_int, (unsigned long long)tt);
    __threadfence();
    last = (atomicAdd(&ctl->done_blocks, 1u) == nblocks - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    volatile Control* vc = ctl;
    const double Tf = vc->T_f, T2 = vc->T2_f;
    for (int c = 0; c < NS3; ++c) r->estimate[c] = vc->est[c] / Tf;
    r->ess = Tf * Tf / T2;
    if (kind == 1) {
      r->max_loglik = ord_decode(vc->max_ll);
    } else {
      const unsigned long long e = vc->max_llq;
      r->max_loglik = e == 0ull ? -INFINITY : (double)llq_dec(e) * (1.0 / 4294967296.0);
    }
    r->sum_wtilde = Tf;
    r->n_particles = N;
    r->n_bins = kind == 1 ? (int64_t)vc->nocc : 0;
    r->kind = kind;
    if (vc->T_int <= 0) atomicOr(&ctl->err, (unsigned)PCSIR_DERR_ZEROSUM);
  }
}

__global__ void __launch_bounds__(R3_THREADS) k_binred3(StepBuffers b, pcsir3_result* r, int64_t N, int sq) {
  const unsigned B = b.ctl->nocc;
  const unsigned need = (B + blockDim.x - 1) / blockDim.x;
  const unsigned active = need < 1u ? 1u : (need < gridDim.x ? need : gridDim.x);
  if (blockIdx.x >= active) return;
  const double m = ord_decode(b.ctl->max_ll);
  const int64_t bs = b.bin_stride;
  Red3 a{};
  for (unsigned bi = blockIdx.x * blockDim.x + threadIdx.x; bi < B; bi += gridDim.x * blockDim.x) {
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
#pragma unroll
    for (int c = 0; c < NS3; ++c) a.est[c] += n * wt * b.dummy[c * bs + bi];
  }
  commit3(a, b, r, N, 1, active);
}

// ---------------------------------------------------------------------------
// SIR in 3D: propagate and the likelihood of every particle (a warp per
// particle), then per-particle weights
// ---------------------------------------------------------------------------
constexpr int S3_THREADS = 256;

__global__ void __launch_bounds__(S3_THREADS)
k_sir3_prop_lik(StepBuffers b, const float* __restrict__ st, const float* __restrict__ nz, int64_t N, Lik3 lp,
                const float* __restrict__ vol, int W, int H, int D, int keep) {
  constexpr int NW = S3_THREADS / 32;
  __shared__ float scratch[NW][2 * (3 * MAXP3)];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* __restrict__ prop = static_cast<float*>(b.prop);
  long long mymax = LLQ_NONE;
  for (int64_t i = (int64_t)blockIdx.x * NW + w; i < N; i += (int64_t)gridDim.x * NW) {
    float v[NS3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      v[p] = __fadd_rn(__fadd_rn(st[p * N + i], st[(3 + p) * N + i]), nz[p * N + i]);
      v[3 + p] = __fadd_rn(st[(3 + p) * N + i], nz[(3 + p) * N + i]);
    }
    v[6] = __fadd_rn(st[6 * N + i], nz[6 * N + i]);
    if (lane < NS3) prop[lane * N + i] = v[lane];
    const LLSum s = warp_loglik3(vol, W, H, D, pos3(v[0], v[1], v[2], v[6]), lp, scratch[w]);
    const long long q = llq_of(s);
    if (lane == 0) {
      b.llq[i] = q;
      if ((keep & PCSIR_KEEP_LOGLIK) && b.ll) b.ll[i] = ll_to_double(s);
    }
    mymax = q > mymax ? q : mymax;
  }
  __shared__ long long red[NW];
  if (lane == 0) red[w] = mymax;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = LLQ_NONE;
    for (int j = 0; j < NW; ++j) m = red[j] > m ? red[j] : m;
    if (m != LLQ_NONE) atomicMax(&b.ctl->max_llq, llq_enc(m));
  }
}

__global__ void __launch_bounds__(R3_THREADS) k_sir3_w(StepBuffers b, pcsir3_result* r, int64_t N, int sq) {
  const unsigned long long me = b.ctl->max_llq;
  const long long mq = llq_dec(me);
  const float* __restrict__ prop = static_cast<const float*>(b.prop);
  kahan kt, k2, ke[NS3];
  long long tint = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const df wd = me == 0ull ? df{0.0f, 0.0f} : wtilde_q(b.llq[i], mq);
    const float wt = wd.hi;
    tint += q_of_wtilde(wd, sq);
    kt.add(wt);
    k2.add(wt * wt);
#pragma unroll
    for (int c = 0; c < NS3; ++c) ke[c].add(wt * prop[c * N + i]);
  }
  Red3 a;
  a.Tf = (double)kt.s - (double)kt.c;
  a.T2 = (double)k2.s - (double)k2.c;
#pragma unroll
  for (int c = 0; c < NS3; ++c) a.est[c] = (double)ke[c].s - (double)ke[c].c;
  a.Tint = tint;
  commit3(a, b, r, N, 0, gridDim.x);
}

}  // namespace pcsir

using namespace pcsir;

struct pcsir3_ctx {
  pcsir3_config cfg{};
  int num_sms = 0;
  StepBuffers b{};
  int32_t* bin_xyz = nullptr;
  pcsir3_result* dres3 = nullptr;
  pcsir3_result* host_res = nullptr;
  Lik3 lik{};
  std::vector<void*> allocs;
  std::string err = "no error";
  bool failed = false;
  int last_kind = -1;
  int64_t last_N = 0;
  int pb_per_sm = 1;
  // attached likelihood surrogate (3D geometry): per-step held-out list and statistics
  SurStep sur{};
  bool sur_on = false;
  bool sur_ran = false;
  unsigned long long sur_steps = 0;
  double psf_sigma_xy = 0.0;
};

namespace {

pcsir_status fail3(pcsir3_ctx* c, pcsir_status st, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (st == PCSIR_ECUDA) c->failed = true;
  }
  return st;
}
pcsir_status cuda_fail3(pcsir3_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail3(c, PCSIR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
bool alloc3(pcsir3_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return true;
}

void free3(pcsir3_ctx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->host_res) cudaFreeHost(c->host_res);
  c->host_res = nullptr;
}

pcsir_status check3(pcsir3_ctx* c, const float* state, int64_t N, const float* vol, int32_t W, int32_t H, int32_t D,
                    const float* noise, double u0) {
  if (!c) return PCSIR_EINVAL;
  if (c->failed) return fail3(c, PCSIR_ESTATE, "context failed earlier: " + c->err);
  if (!state || !vol || !noise) return fail3(c, PCSIR_EINVAL, "state, volume and noise must be device pointers");
  if (N < 1) return fail3(c, PCSIR_EINVAL, "N must be >= 1");
  if (N > c->cfg.max_particles) return fail3(c, PCSIR_ERANGE, "N exceeds max_particles of the context");
  if (W < 1 || H < 1 || D < 1) return fail3(c, PCSIR_EINVAL, "volume sizes must be >= 1");
  if (!(u0 >= 0.0 && u0 < 1.0)) return fail3(c, PCSIR_EINVAL, "u0 must lie in [0, 1)");
  return PCSIR_OK;
}

pcsir_status finish3(pcsir3_ctx* c, cudaStream_t s, pcsir3_result* out, int kind, int64_t N) {
  cudaError_t e = cudaMemcpyAsync(c->host_res, c->dres3, sizeof(pcsir3_result), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && out && out != c->host_res)
    e = cudaMemcpyAsync(out, c->dres3, sizeof(pcsir3_result), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail3(c, e, "copy of step result");
  c->last_kind = kind;
  c->last_N = N;
  return PCSIR_OK;
}

}  // namespace

extern "C" {

const char* pcsir3_last_error(pcsir3_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

pcsir_status pcsir3_create(const pcsir3_config* cfg, pcsir3_ctx** out) {
  if (!out) return PCSIR_EINVAL;
  *out = nullptr;
  if (!cfg) return PCSIR_EINVAL;
  if (cfg->patch_xy < 1 || cfg->patch_xy > MAXP3 || (cfg->patch_xy & 1) == 0 || cfg->patch_z < 1 ||
      cfg->patch_z > MAXP3 || (cfg->patch_z & 1) == 0 || cfg->reserved != 0)
    return PCSIR_EINVAL;
  if (!(cfg->psf_sigma_xy > 0.0) || !(cfg->psf_sigma_z > 0.0) || !(cfg->bg > 0.0) || !std::isfinite(cfg->bg) ||
      !std::isfinite(cfg->psf_sigma_xy) || !std::isfinite(cfg->psf_sigma_z))
    return PCSIR_EINVAL;
  if (cfg->max_particles < 1 || cfg->max_particles > MAX_PARTICLES) return PCSIR_EINVAL;
  if (cfg->keep & ~(PCSIR_KEEP_ANCESTORS | PCSIR_KEEP_WEIGHTS | PCSIR_KEEP_PARTICLE_BIN | PCSIR_KEEP_LOGLIK |
                    PCSIR_KEEP_QWEIGHTS))
    return PCSIR_EINVAL;
  pcsir3_ctx* c = new (std::nothrow) pcsir3_ctx();
  if (!c) return PCSIR_ENOMEM;
  c->cfg = *cfg;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return PCSIR_ECUDA;
  }
  const int64_t nmax = cfg->max_particles;
  int hbits = 10;
  while ((int64_t(1) << hbits) < 2 * nmax) ++hbits;
  const size_t hcap = size_t(1) << hbits;
  StepBuffers& b = c->b;
  b.hbits = hbits;
  b.bin_stride = nmax;
  b.max_tiles = (nmax + SCAN_TILE - 1) / SCAN_TILE;
  bool ok = alloc3(c, &b.hkey, hcap) && alloc3(c, &b.hcnt, hcap) && alloc3(c, &b.hsum, (size_t)NS3 * hcap) &&
            alloc3(c, &b.hrank, hcap) && alloc3(c, &b.hq, hcap) && alloc3(c, &b.hw, hcap) &&
            alloc3(c, &b.occ, (size_t)nmax) && alloc3(c, &c->bin_xyz, 3 * (size_t)nmax) &&
            alloc3(c, &b.bin_cnt, (size_t)nmax) && alloc3(c, &b.dummy, (size_t)NS3 * nmax) &&
            alloc3(c, &b.bin_ll, (size_t)nmax) && alloc3(c, &b.pslot, (size_t)nmax) && alloc3(c, &b.llq, (size_t)nmax) &&
            alloc3(c, &b.tile_sum, (size_t)b.max_tiles) && alloc3(c, &b.tile_excl, (size_t)b.max_tiles) &&
            alloc3(c, &b.tile_lo, (size_t)b.max_tiles + 1) && alloc3(c, &b.tile_ovx, (size_t)b.max_tiles + 1) &&
            alloc3(c, &b.ctl, 1) && alloc3(c, &b.dres, 1) && alloc3(c, &c->dres3, 1);
  if (ok) {
    float* p = nullptr;
    ok = alloc3(c, &p, (size_t)NS3 * nmax);
    b.prop = p;
  }
  if (ok && (cfg->keep & PCSIR_KEEP_ANCESTORS)) ok = alloc3(c, &b.anc, (size_t)nmax);
  if (ok && (cfg->keep & PCSIR_KEEP_WEIGHTS)) ok = alloc3(c, &b.wout, (size_t)nmax);
  if (ok && (cfg->keep & PCSIR_KEEP_QWEIGHTS)) ok = alloc3(c, &b.qout, (size_t)nmax);
  if (ok && (cfg->keep & PCSIR_KEEP_PARTICLE_BIN)) ok = alloc3(c, &b.pbin, (size_t)nmax);
  if (ok && (cfg->keep & PCSIR_KEEP_LOGLIK)) ok = alloc3(c, &b.ll, (size_t)nmax);
  if (!ok) {
    free3(c);
    delete c;
    return PCSIR_ENOMEM;
  }
  b.derr_out = &c->dres3->device_error;
  const size_t smem = sizeof(Local3);
  e = cudaFuncSetAttribute(k_prop_bin3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->pb_per_sm, k_prop_bin3, P3_THREADS, smem);
  if (c->pb_per_sm < 1) c->pb_per_sm = 1;
  if (e == cudaSuccess) e = prepare_resample();
  if (e == cudaSuccess) e = cudaMallocHost(&c->host_res, sizeof(pcsir3_result));
  if (e == cudaSuccess) e = cudaMemset(b.hkey, 0xff, hcap * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(b.hcnt, 0, hcap * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(b.hsum, 0, (size_t)NS3 * hcap * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(c->dres3, 0, sizeof(pcsir3_result));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    free3(c);
    delete c;
    return e == cudaErrorMemoryAllocation ? PCSIR_ENOMEM : PCSIR_ECUDA;
  }
  std::memset(c->host_res, 0, sizeof(pcsir3_result));
  c->psf_sigma_xy = cfg->psf_sigma_xy;
  Lik3& lp = c->lik;
  lp.Pxy = cfg->patch_xy;
  lp.Pz = cfg->patch_z;
  lp.bg = (float)cfg->bg;
  const double cxy = 1.0 / (2.0 * cfg->psf_sigma_xy * cfg->psf_sigma_xy);
  const double cz = 1.0 / (2.0 * cfg->psf_sigma_z * cfg->psf_sigma_z);
  lp.c2xy = {(float)cxy, (float)(cxy - (double)(float)cxy)};
  lp.c2z = {(float)cz, (float)(cz - (double)(float)cz)};
  *out = c;
  return PCSIR_OK;
}

pcsir_status pcsir3_destroy(pcsir3_ctx* ctx) {
  if (!ctx) return PCSIR_OK;
  cudaDeviceSynchronize();
  free3(ctx);
  delete ctx;
  return PCSIR_OK;
}

pcsir_status pcsir3_step(pcsir3_ctx* ctx, float* state, int64_t N, const float* volume, int32_t W, int32_t H,
                         int32_t D, double hx, double hy, double hz, const float* noise, double u0, void* stream,
                         pcsir3_result* result_host) {
  pcsir_status st = check3(ctx, state, N, volume, W, H, D, noise, u0);
  if (st != PCSIR_OK) return st;
  if (!(hx > 0.0 && hx <= MAX_H && hy > 0.0 && hy <= MAX_H && hz > 0.0 && hz <= MAX_H))
    return fail3(ctx, PCSIR_EINVAL, "cell edges must lie in (0, 8]");
  if (ctx->sur_on && (int64_t)W * H * D > sur_max_pixels(ctx->sur.sur))
    return fail3(ctx, PCSIR_ERANGE, "volume larger than the surrogate's max_pixels");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const StepBuffers& b = ctx->b;
  cudaError_t e = cudaMemsetAsync(b.ctl, 0, sizeof(Control), s);
  if (e != cudaSuccess) return cuda_fail3(ctx, e, "reset of step control block");
  const long long hqx = llrint(hx * 2147483648.0), hqy = llrint(hy * 2147483648.0), hqz = llrint(hz * 2147483648.0);
  const int64_t nchunks = (N + P3_CHUNK - 1) / P3_CHUNK;
  const int grid = (int)std::min<int64_t>(nchunks, (int64_t)ctx->num_sms * ctx->pb_per_sm);
  k_prop_bin3<<<grid, P3_THREADS, sizeof(Local3), s>>>(b, state, noise, N, (float)hx, (float)hy, (float)hz, hqx, hqy,
                                                       hqz);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    if (!ctx->sur_on) {
      k_bins3<false><<<ctx->num_sms * 4, B3_THREADS, 0, s>>>(b, ctx->bin_xyz, ctx->lik, volume, W, H, D, hqx, hqy,
                                                             hqz, SurBins3{});
      e = cudaGetLastError();
    } else {
      SurStep sp = ctx->sur;
      sp.salt = ctx->sur_steps;
      const SurBins3 sb{sp.salt, sp.frac, sp.min_holdout, sp.ho_cap, sp.ho_bin, sp.ho_ll, sp.stats};
      e = cudaMemsetAsync(sp.stats, 0, sizeof(SurStats), s);
      if (e == cudaSuccess) {
        k_bins3<true><<<ctx->num_sms * 4, B3_THREADS, 0, s>>>(b, ctx->bin_xyz, ctx->lik, volume, W, H, D, hqx, hqy,
                                                              hqz, sb);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = launch_sur_step3(sp, b, ctx->cfg.bg, ctx->psf_sigma_xy, volume, W, H, D, s);
      if (e == cudaSuccess) {
        k_bins3_fallback<<<ctx->num_sms * 4, B3_THREADS, 0, s>>>(b, ctx->lik, volume, W, H, D, sp.stats);
        e = cudaGetLastError();
      }
      ctx->sur_steps++;
    }
  }
  ctx->sur_ran = ctx->sur_on;
  if (e == cudaSuccess) {
    k_binred3<<<ctx->num_sms * 2, R3_THREADS, 0, s>>>(b, ctx->dres3, N, weight_scale_bits(N));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_resample7(b, state, N, u0, WSRC_BINS, ctx->cfg.keep, s);
  if (e != cudaSuccess) return cuda_fail3(ctx, e, "3D pcSIR kernels");
  return finish3(ctx, s, result_host, 1, N);
}

pcsir_status sir3_step(pcsir3_ctx* ctx, float* state, int64_t N, const float* volume, int32_t W, int32_t H,
                       int32_t D, const float* noise, double u0, void* stream, pcsir3_result* result_host) {
  pcsir_status st = check3(ctx, state, N, volume, W, H, D, noise, u0);
  if (st != PCSIR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const StepBuffers& b = ctx->b;
  cudaError_t e = cudaMemsetAsync(b.ctl, 0, sizeof(Control), s);
  if (e != cudaSuccess) return cuda_fail3(ctx, e, "reset of step control block");
  const int64_t want = (N + S3_THREADS / 32 - 1) / (S3_THREADS / 32);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->num_sms * 16));
  k_sir3_prop_lik<<<grid, S3_THREADS, 0, s>>>(b, state, noise, N, ctx->lik, volume, W, H, D, ctx->cfg.keep);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    const int rgrid = (int)std::min<int64_t>((N + R3_THREADS - 1) / R3_THREADS, (int64_t)ctx->num_sms * 4);
    k_sir3_w<<<rgrid, R3_THREADS, 0, s>>>(b, ctx->dres3, N, weight_scale_bits(N));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = launch_resample7(b, state, N, u0, WSRC_PARTICLES, ctx->cfg.keep & ~PCSIR_KEEP_PARTICLE_BIN, s);
  if (e != cudaSuccess) return cuda_fail3(ctx, e, "3D SIR kernels");
  return finish3(ctx, s, result_host, 0, N);
}

pcsir_status pcsir3_get_outputs(pcsir3_ctx* ctx, pcsir3_outputs* o) {
  if (!ctx || !o) return PCSIR_EINVAL;
  if (ctx->last_kind < 0) return fail3(ctx, PCSIR_ESTATE, "no step has run on this context");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail3(ctx, e, "synchronisation");
  std::memset(o, 0, sizeof(*o));
  const StepBuffers& b = ctx->b;
  o->n_particles = ctx->last_N;
  o->n_bins = ctx->last_kind == 1 ? ctx->host_res->n_bins : 0;
  o->bin_stride = b.bin_stride;
  o->prop_state = static_cast<const float*>(b.prop);
  if (ctx->last_kind == 1) {
    o->bin_xyz = ctx->bin_xyz;
    o->bin_count = b.bin_cnt;
    o->dummy = b.dummy;
    o->bin_loglik = b.bin_ll;
    o->particle_bin = b.pbin;
  } else {
    o->loglik = b.ll;
  }
  o->ancestor = b.anc;
  o->weight = b.wout;
  o->qweight = reinterpret_cast<const int64_t*>(b.qout);
  return PCSIR_OK;
}

pcsir_status pcsir3_attach_surrogate(pcsir3_ctx* ctx, pcsir_surrogate* sur, double holdout_frac, int32_t min_holdout,
                                     double window, double max_err) {
  if (!ctx) return PCSIR_EINVAL;
  if (ctx->failed) return fail3(ctx, PCSIR_ESTATE, "context failed earlier: " + ctx->err);
  if (!sur) {
    ctx->sur_on = false;
    return PCSIR_OK;
  }
  if (!(holdout_frac >= 0.0 && holdout_frac <= 1.0) || min_holdout < 0 || !(window >= 0.0) || !(max_err >= 0.0))
    return fail3(ctx, PCSIR_EINVAL, "invalid held-out fraction, window or error threshold");
  if (sur_dim(sur) != 3) return fail3(ctx, PCSIR_EINVAL, "a 2D surrogate attaches to a 2D context");
  if (ctx->cfg.patch_xy != PCSIR_SUR3_PATCH_XY || ctx->cfg.patch_z != PCSIR_SUR3_PATCH_Z)
    return fail3(ctx, PCSIR_EINVAL, "the 3D surrogate models an 11 x 11 x 7 patch");
  SurStep& sp = ctx->sur;
  if (!sp.stats) {
    constexpr int HO_CAP = 1 << 16;
    if (!(alloc3(ctx, &sp.ho_bin, HO_CAP) && alloc3(ctx, &sp.ho_ll, HO_CAP) && alloc3(ctx, &sp.stats, 1))) {
      sp.stats = nullptr;
      return fail3(ctx, PCSIR_ENOMEM, "held-out list allocation");
    }
    sp.ho_cap = HO_CAP;
    const cudaError_t e = cudaMemset(sp.stats, 0, sizeof(SurStats));
    if (e != cudaSuccess) return cuda_fail3(ctx, e, "held-out statistics");
  }
  sp.sur = sur;
  sp.frac = holdout_frac;
  sp.min_holdout = min_holdout;
  sp.window = window;
  sp.max_err = max_err;
  ctx->sur_on = true;
  ctx->sur_steps = 0;
  return PCSIR_OK;
}

pcsir_status pcsir3_surrogate_last_check(pcsir3_ctx* ctx, pcsir_surrogate_check* out) {
  if (!ctx || !out) return PCSIR_EINVAL;
  if (!ctx->sur_ran || ctx->last_kind != 1) return fail3(ctx, PCSIR_ESTATE, "the last step did not use a surrogate");
  SurStats st{};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&st, ctx->sur.stats, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail3(ctx, e, "reading surrogate statistics");
  std::memset(out, 0, sizeof(*out));
  const int64_t nb = ctx->host_res->n_bins;
  const int64_t nho = std::min<int64_t>(st.n_ho, ctx->sur.ho_cap);
  out->n_dummies = nb;
  out->n_holdout = nho;
  out->n_significant = st.n_sig;
  out->n_clipped = st.n_clipped;
  out->fallback = st.fallback ? 1 : 0;
  out->n_exact = st.fallback ? nb : (int64_t)st.n_ho + (int64_t)st.n_clipped;
  out->max_abs_err = st.max_err;
  out->rms_err = nho > 0 ? std::sqrt(st.sum_sq / (double)nho) : 0.0;
  return PCSIR_OK;
}

pcsir_status pcsir3_last_result(pcsir3_ctx* ctx, pcsir3_result* out) {
  if (!ctx || !out) return PCSIR_EINVAL;
  std::memcpy(out, ctx->host_res, sizeof(*out));
  return PCSIR_OK;
}

}  // extern "C"
