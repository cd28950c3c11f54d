// ESS-thresholded SIR and pcSIR steps (Algorithms 1 and 2 with their test on
// the effective sample size, Section 3: resampling happens only when N_eff
// falls below N_thr): the particles carry log-weights from step to step until
// the test resamples them.
//
// The carried log-weights are int64 fixed point (units of 2^-32), the form in
// which SIR's per-particle log-likelihoods already enter the integer weights of
// the resampling kernel; adding a step's log-likelihood is an exact integer
// addition.  pcSIR with carried weights needs each cell's centre of mass
// weighted by w_{k-1} (Section 4 forms it from the states and their weights):
//
//   k_ess_rank   bin index of every occupied hash slot; zeroes the per-bin sums
//   k_ess_cellmax per bin: M_b, the largest carried log-weight of its members
//                rounded down to a whole nat
//   k_ess_wsums  per bin: sum of w_i and of w_i (s_i - r_b) for every state
//                component, w_i = exp(logw_i 2^-32 - M_b): weights relative to
//                the cell's own largest (a common factor of the cell's sums,
//                so the weighted mean is unchanged, and no cell's weights all
//                underflow in FP32 however far below the global maximum they
//                lie), r_b the cell's lower corner for x, y and the step's
//                anchors (particle 0's input values) for vx, vy, I0.  FP32
//                products summed in shared memory over rounds of ESS_ROUND
//                particles, then added into FP64 per-bin sums.
//   k_ess_bins   weighted dummy r_b + S_b / W_b (the plain mean when W_b = 0),
//                or the cell centre for x, y with pcSIR-CoC, and its
//                likelihood; the hash slots return to empty
//   k_ess_lw     logw_i + ll_{bin(i)} in fixed point, and its maximum
//
// then the usual per-particle weight reduction (ESS, posterior mean) and the
// resampling kernel, which decides on the device whether to resample.
#include <algorithm>

#include "pcsir_device.cuh"

namespace pcsir {

LikParams make_lik(const ModelParams& m);  // pcsir_kernels.cu

constexpr int ESS_THREADS = 256;
constexpr int ESS_SMEM_BINS = 2048;  // bins whose sums a block keeps in shared memory
constexpr int ESS_WARP_BINS = 256;   // up to this many bins, each warp keeps its own copy
constexpr int ESS_ROUND = 8192;      // particles per shared-memory round of a block
constexpr int ESS_BIN_WARPS = ESS_THREADS / 32;
constexpr int ESS_MAXP = 127;        // largest patch side

// exp(l 2^-32 - m) for a fixed-point log-weight l and a whole-nat reference m >= floor(l 2^-32).
// The exponent is formed from two 32-bit conversions (the 64-bit conversion runs on the FP64 pipe),
// the whole nats in 64-bit integers so that no difference overflows
__device__ __forceinline__ float rel_weight(long long l, int m) {
  const long long dh = (l >> 32) - (long long)m;  // whole nats below the reference, <= 0
  if (dh < -200) return 0.0f;                     // below FP32's range
  return expf((float)dh + (float)(unsigned)(l & 0xffffffffll) * 2.3283064365386963e-10f);
}

// lower corner of cell b along one axis, the reference of the weighted position offsets
__device__ __forceinline__ float cell_ref(int b, float h) { return __fsub_rn(__fmul_rn((float)b, h), 0.5f); }

__device__ __forceinline__ float anchor_f(const Control* ctl, int c) {
  return (float)((double)ctl->anchor[2 + c] * VAL_INV);
}

// M_b per bin, in whole nats (INT_MIN: no member carries weight); it occupies the per-bin count
// array, which k_ess_bins fills only afterwards
__device__ __forceinline__ int* cell_max(const StepBuffers& b) { return reinterpret_cast<int*>(b.bin_cnt); }

__global__ void __launch_bounds__(ESS_THREADS) k_ess_rank(StepBuffers b) {
  const unsigned B = b.ctl->nocc;
  const int64_t bs = b.bin_stride;
  for (unsigned bi = blockIdx.x * blockDim.x + threadIdx.x; bi < B; bi += gridDim.x * blockDim.x) {
    b.hrank[b.occ[bi]] = bi;
    b.bin_ll[bi] = 0.0;  // sum of the members' weights until k_ess_bins
    cell_max(b)[bi] = INT_MIN;
#pragma unroll
    for (int c = 0; c < 5; ++c) b.dummy[c * bs + bi] = 0.0;
  }
}

__global__ void __launch_bounds__(ESS_THREADS) k_ess_cellmax(StepBuffers b, const long long* __restrict__ lw,
                                                             int64_t N) {
  // per block in shared memory when the bins fit (then one global atomic per bin and block), else
  // straight into the global array, where the lanes of one bin first agree across the warp
  __shared__ int smax[ESS_SMEM_BINS];
  const unsigned B = b.ctl->nocc;
  const bool local = B <= (unsigned)ESS_SMEM_BINS;
  int* __restrict__ gmax = cell_max(b);
  if (local) {
    for (unsigned j = threadIdx.x; j < B; j += blockDim.x) smax[j] = INT_MIN;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t stride = 4 * (int64_t)gridDim.x * blockDim.x;
  // four particles per thread and pass, their loads and gathers issued first; the loop bound is
  // uniform over the warp (the warp-wide match and shuffles need every lane)
  for (int64_t w0 = 4 * (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < N; w0 += stride) {
    unsigned cell[4];
    int v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = w0 + lane + (int64_t)k * blockDim.x;
      cell[k] = 0xffffffffu;
      v[k] = INT_MIN;
      if (i >= N) continue;
      const unsigned bi = b.hrank[b.pslot[i]];
      const long long l = lw[i];
      if (bi < B && l != LLQ_NONE) {
        cell[k] = bi;
        v[k] = (int)(l >> 32);  // floor of the log-weight in nats
      }
    }
    if (local) {  // 32-bit shared atomics settle equal addresses within the warp themselves
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (cell[k] != 0xffffffffu) atomicMax(&smax[cell[k]], v[k]);
      continue;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned peers = __match_any_sync(0xffffffffu, cell[k]);
      unsigned rem = peers & ~(1u << lane);
      const unsigned steps = __reduce_max_sync(0xffffffffu, (unsigned)__popc(rem));
      int m = v[k];
      for (unsigned st = 0; st < steps; ++st) {
        const int src = rem ? __ffs(rem) - 1 : lane;
        rem &= rem - 1u;
        m = max(m, __shfl_sync(0xffffffffu, v[k], src));
      }
      if (cell[k] != 0xffffffffu && (peers & ((1u << lane) - 1u)) == 0u) atomicMax(&gmax[cell[k]], m);
    }
  }
  if (local) {
    __syncthreads();
    for (unsigned j = threadIdx.x; j < B; j += blockDim.x)
      if (smax[j] != INT_MIN) atomicMax(&gmax[j], smax[j]);
  }
}

__global__ void __launch_bounds__(ESS_THREADS) k_ess_wsums(StepBuffers b, const long long* __restrict__ lw,
                                                           int64_t N, float h) {
  // sums in shared memory: with few cells (B <= ESS_WARP_BINS) one copy per warp, so that only the
  // lanes of one warp meet on an address; else one copy per block (B <= ESS_SMEM_BINS); else the
  // FP64 per-bin sums in global memory directly
  __shared__ float acc[6 * ESS_SMEM_BINS];
  const unsigned B = b.ctl->nocc;
  const bool per_warp = B <= (unsigned)ESS_WARP_BINS;
  const bool local = B <= (unsigned)ESS_SMEM_BINS;
  const unsigned nslots = per_warp ? (unsigned)(ESS_THREADS / 32 * 6 * ESS_WARP_BINS) : 6u * B;
  const unsigned stride = per_warp ? (unsigned)ESS_WARP_BINS : B;  // between the six sums of a copy
  float* mine = per_warp ? acc + (threadIdx.x >> 5) * 6 * ESS_WARP_BINS : acc;
  const float* __restrict__ prop = static_cast<const float*>(b.prop);
  const int* __restrict__ cmax = cell_max(b);
  const int64_t bs = b.bin_stride;
  float anc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) anc[c] = anchor_f(b.ctl, c);
  if (local) {
    for (unsigned j = threadIdx.x; j < nslots; j += blockDim.x) acc[j] = 0.0f;
  }
  __syncthreads();
  // a contiguous range of particles per block, in rounds of ESS_ROUND
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per;
  const int64_t hi = lo + per < N ? lo + per : N;
  const int lane = threadIdx.x & 31;
  for (int64_t r0 = lo; r0 < hi; r0 += ESS_ROUND) {
    const int64_t r1 = r0 + ESS_ROUND < hi ? r0 + ESS_ROUND : hi;
    // four particles per thread and pass, their loads and gathers issued before the sums; the
    // loop bound is uniform over the warp (the warp-wide match and shuffles below need every lane)
    for (int64_t w0 = r0 + (threadIdx.x & ~31); w0 < r1; w0 += 4 * (int64_t)blockDim.x) {
      unsigned bi[4];
      float w[4], d[4][5];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t i = w0 + lane + (int64_t)k * blockDim.x;
        bi[k] = 0xffffffffu;
        w[k] = 0.0f;
#pragma unroll
        for (int c = 0; c < 5; ++c) d[k][c] = 0.0f;
        if (i >= r1) continue;
        const unsigned g = b.pslot[i];
        bi[k] = b.hrank[g];
        const unsigned long long key = b.hkey[g];
        const long long l = lw[i];
        // relative to the cell's largest carried log-weight (bi < B whenever l carries weight)
        w[k] = l == LLQ_NONE || bi[k] >= B ? 0.0f : rel_weight(l, cmax[bi[k]]);
        d[k][0] = prop[i] - cell_ref(key_bx(key), h);
        d[k][1] = prop[N + i] - cell_ref(key_by(key), h);
#pragma unroll
        for (int c = 0; c < 3; ++c) d[k][2 + c] = prop[(2 + c) * N + i] - anc[c];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        // lanes of one cell first add their terms across the warp (the lowest lane of the cell
        // gathers the others' in lane order), so that an accumulator sees one atomic per cell
        // and warp instruction; past the range, or after a failed cell insertion
        // (PCSIR_DERR_RANGE), bi >= B and the lane adds nothing
        const unsigned cell = bi[k] < B ? bi[k] : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, cell);
        const unsigned others = peers & ~(1u << lane);
        const unsigned steps = __reduce_max_sync(0xffffffffu, (unsigned)__popc(others));
        float v[6] = {w[k], w[k] * d[k][0], w[k] * d[k][1], w[k] * d[k][2], w[k] * d[k][3], w[k] * d[k][4]};
        float t[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) t[a] = v[a];
        unsigned rem = others;
        for (unsigned st = 0; st < steps; ++st) {
          const int src = rem ? __ffs(rem) - 1 : lane;
          rem &= rem - 1u;
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            const float x = __shfl_sync(0xffffffffu, v[a], src);
            if (src != lane) t[a] += x;
          }
        }
        if (cell == 0xffffffffu || (peers & ((1u << lane) - 1u)) != 0u) continue;
        if (local) {
#pragma unroll
          for (int a = 0; a < 6; ++a) atomicAdd(&mine[a * stride + cell], t[a]);
        } else {
          atomicAdd(&b.bin_ll[cell], (double)t[0]);
#pragma unroll
          for (int c = 0; c < 5; ++c) atomicAdd(&b.dummy[c * bs + cell], (double)t[1 + c]);
        }
      }
    }
    if (local) {
      __syncthreads();
      const unsigned ncopies = per_warp ? (unsigned)(ESS_THREADS / 32) : 1u;
      for (unsigned j = threadIdx.x; j < B; j += blockDim.x) {
        float t[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        for (unsigned cp = 0; cp < ncopies; ++cp) {
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            float* slot = acc + cp * 6 * stride + a * stride + j;
            t[a] += *slot;
            *slot = 0.0f;
          }
        }
        if (t[0] != 0.0f) {
          atomicAdd(&b.bin_ll[j], (double)t[0]);
#pragma unroll
          for (int c = 0; c < 5; ++c) atomicAdd(&b.dummy[c * bs + j], (double)t[1 + c]);
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(ESS_THREADS) k_ess_bins(StepBuffers b, LikParams lp, const float* __restrict__ img,
                                                          int W, int H, float h, long long hq, int coc) {
  __shared__ float scratch[ESS_BIN_WARPS][4 * ESS_MAXP];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const unsigned B = b.ctl->nocc;
  const size_t hcap = size_t(1) << b.hbits;
  const int64_t bs = b.bin_stride;
  double mymax = -INFINITY;
  for (unsigned bi = blockIdx.x * ESS_BIN_WARPS + wp; bi < B; bi += gridDim.x * ESS_BIN_WARPS) {
    const unsigned g = b.occ[bi];
    const unsigned long long key = b.hkey[g];
    const int bx = key_bx(key), by = key_by(key);
    const unsigned n = b.hcnt[g];
    const double wsum = b.bin_ll[bi];
    double dum[5];
    if (wsum > 0.0) {
      dum[0] = (double)cell_ref(bx, h) + b.dummy[bi] / wsum;
      dum[1] = (double)cell_ref(by, h) + b.dummy[bs + bi] / wsum;
#pragma unroll
      for (int c = 0; c < 3; ++c) dum[2 + c] = (double)anchor_f(b.ctl, c) + b.dummy[(2 + c) * bs + bi] / wsum;
    } else {  // no member carries weight: the plain mean from the exact sums
      const double dn = (double)n;
      const double rdn = 1.0 / dn;  // one FP64 division per cell (GB300's FP64 rate is low)
      dum[0] = ((double)((long long)bx * hq) + (double)b.hsum[g] * rdn) * POS_INV;
      dum[1] = ((double)((long long)by * hq) + (double)b.hsum[hcap + g] * rdn) * POS_INV;
#pragma unroll
      for (int c = 2; c < 5; ++c) dum[c] = ((double)b.ctl->anchor[c] + (double)b.hsum[c * hcap + g] * rdn) * VAL_INV;
    }
    if (coc) {  // pcSIR-CoC: the cell's geometric centre
      dum[0] = ((double)bx + 0.5) * (double)h - 0.5;
      dum[1] = ((double)by + 0.5) * (double)h - 0.5;
    }
    __syncwarp();
    const LLSum ls = warp_loglik(img, W, H, lik_pos(dum[0], dum[1], dum[4]), lp, scratch[wp]);
    const double ll = ls.bad ? -INFINITY : ll_to_double(ls);
    __syncwarp();
    if (lane == 0) {
      if (ls.bad) raise_flag(b.ctl, PCSIR_DERR_NONFINITE);
#pragma unroll
      for (int c = 0; c < 5; ++c) b.dummy[c * bs + bi] = dum[c];
      b.bin_ll[bi] = ll;
      b.bin_cnt[bi] = n;
      b.bin_xy[bi] = bx;
      b.bin_xy[bs + bi] = by;
      b.hq[g] = llq_of(ls);  // the cell's fixed-point log-likelihood, read per particle next
      b.hkey[g] = EMPTY_KEY;
      b.hcnt[g] = 0u;
#pragma unroll
      for (int c = 0; c < 5; ++c) b.hsum[c * hcap + g] = 0;
    }
    mymax = fmax(mymax, ll);
  }
  // maximum over the dummies (reported only; the weights use the particles' maximum)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mymax = fmax(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
  if (lane == 0 && mymax > -INFINITY) atomicMax(&b.ctl->max_ll, ord_encode(mymax));
}

__device__ __forceinline__ void ess_block_max(long long v, Control* ctl) {
  __shared__ long long red[ESS_THREADS / 32];
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

// logw_i + ll_i: from the particle's cell (pcSIR, PCSIR = true) or from SIR's per-particle
// values already in b.llq; INT64_MIN (no weight) on either side stays INT64_MIN
template <bool PCSIR>
__global__ void __launch_bounds__(ESS_THREADS) k_ess_lw(StepBuffers b, const long long* __restrict__ lw, int64_t N) {
  long long m = LLQ_NONE;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const long long l = PCSIR ? b.hq[b.pslot[i]] : b.llq[i];
    const long long p = lw[i];
    const long long v = (l == LLQ_NONE || p == LLQ_NONE) ? LLQ_NONE : p + l;
    b.llq[i] = v;
    if (PCSIR && b.pbin) b.pbin[i] = b.hrank[b.pslot[i]];
    m = v > m ? v : m;
  }
  ess_block_max(m, b.ctl);
}

static int ess_grid(int64_t n, int threads, int num_sms, int per_sm) {
  const int64_t want = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * per_sm));
}

cudaError_t launch_pcsir_ess_front(const StepBuffers& b, const ModelParams& m, const long long* lw_in,
                                   const float* img, int W, int H, int64_t N, double h, int num_sms,
                                   cudaStream_t s) {
  const int full = num_sms * 8;  // blocks of the per-bin kernels (they stop at the device's bin count)
  k_ess_rank<<<full, ESS_THREADS, 0, s>>>(b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ess_cellmax<<<ess_grid(N, 4 * ESS_THREADS, num_sms, 8), ESS_THREADS, 0, s>>>(b, lw_in, N);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_ess_wsums<<<ess_grid(N, ESS_ROUND, num_sms, 4), ESS_THREADS, 0, s>>>(b, lw_in, N, (float)h);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long hq = llrint(h * 2147483648.0);
  k_ess_bins<<<full, ESS_THREADS, 0, s>>>(b, make_lik(m), img, W, H, (float)h, hq, m.coc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_ess_lw<true><<<ess_grid(N, ESS_THREADS, num_sms, 8), ESS_THREADS, 0, s>>>(b, lw_in, N);
  return cudaGetLastError();
}

cudaError_t launch_sir_ess_front(const StepBuffers& b, const long long* lw_in, int64_t N, int num_sms,
                                 cudaStream_t s) {
  // the maximum so far is that of the log-likelihoods alone: start again for the sums
  cudaError_t e = cudaMemsetAsync(&b.ctl->max_llq, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_ess_lw<false><<<ess_grid(N, ESS_THREADS, num_sms, 8), ESS_THREADS, 0, s>>>(b, lw_in, N);
  return cudaGetLastError();
}

}  // namespace pcsir
