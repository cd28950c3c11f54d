// Learned likelihood surrogate of the pcSIR dummy likelihood: the exact
// window term of every window of a frame (box filter), dataset of (inputs,
// residual log-likelihood) rows generated by the method's own steps,
// training (forward, backward and Adam) with the tcgen05 GEMM of
// pcsir_mlp.cu, a fused tcgen05 inference kernel that builds each dummy's
// inputs from the image in shared memory and runs both hidden layers with
// TMEM accumulation, and the held-out check of a surrogate-assisted step.
//
// Network: 445 -> 256 -> 256 -> 1, SiLU.  Device parameter layout (FP32
// master copy, gradients and Adam moments alike): W1 [256][448] (columns 445..447
// stay zero), b1 [256], W2 [256][256], b2 [256], w3 [256], b3; bf16 copies of W1
// and W2 feed the tensor cores.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "pcsir_device.cuh"
#include "pcsir_tc.cuh"

namespace pcsir {

constexpr int SUR_HID = PCSIR_SUR_HIDDEN;  // 256
constexpr int SUR_K1_MAX = 896;            // the largest padded input count (3D)

// Input geometry of a surrogate: the patch and the state features that follow
// it, and the packed parameter layout that depends on the input count.
//   2D: 21 x 21 pixels, then 2 (x - cx), 2 (y - cy), I0 / i0_ref, sigma / sigma_ref: 445 inputs
//   3D: 11 x 11 x 7 voxels, then 2 (x - cx), 2 (y - cy), 2 (z - cz), I0 / i0_ref,
//       sigma_xy / sigma_ref: 852 inputs
// Inputs are padded with zeros to k1, a multiple of 64.
struct SurGeom {
  int dim;
  int px, py, pz;  // patch sides
  int npix, nfeat, nin, k1;
  int irow;        // row of I0 in the dummy array (2D: 4, 3D: 6)
  long long off_w1, off_b1, off_w2, off_b2, off_w3, off_b3, ndev;
};

inline SurGeom make_geom(int dim) {
  SurGeom g{};
  g.dim = dim;
  if (dim == 3) {
    g.px = g.py = PCSIR_SUR3_PATCH_XY;
    g.pz = PCSIR_SUR3_PATCH_Z;
    g.nfeat = 5;
    g.irow = 6;
  } else {
    g.px = g.py = PCSIR_SUR_PATCH;
    g.pz = 1;
    g.nfeat = 4;
    g.irow = 4;
  }
  g.npix = g.px * g.py * g.pz;
  g.nin = g.npix + g.nfeat;
  g.k1 = (g.nin + 63) / 64 * 64;
  g.off_w1 = 0;
  g.off_b1 = g.off_w1 + (long long)SUR_HID * g.k1;
  g.off_w2 = g.off_b1 + SUR_HID;
  g.off_b2 = g.off_w2 + (long long)SUR_HID * SUR_HID;
  g.off_w3 = g.off_b2 + SUR_HID;
  g.off_b3 = g.off_w3 + SUR_HID;
  g.ndev = g.off_b3 + 1;
  return g;
}

// Inputs of one state: patch value f < npix, then the state features.
struct SurFeat {
  float bg, inv_i0ref, sig_feat;
  double inv_i0ref_d;
};

struct SurRowInfo {
  long long base;   // volume offset of the patch's first voxel (smallest x, y, z)
  float feat[4];    // 2D: dx, dy, I0; 3D: dx, dy, dz, I0 (scaled as above)
  int valid;
};

// nearest voxel of a state and whether its whole patch lies inside the W x H x D volume
__device__ __forceinline__ SurRowInfo sur_row_info(const SurGeom& g, const double* dummy, long long stride,
                                                   long long d, int W, int H, int D, const SurFeat& sf) {
  SurRowInfo ri{0, {0.f, 0.f, 0.f, 0.f}, 0};
  const double x = dummy[d], y = dummy[stride + d], i0 = dummy[g.irow * stride + d];
  const int rx = g.px >> 1, ry = g.py >> 1, rz = g.pz >> 1;
  if (g.dim == 2) {
    int cx, cy;
    if (sur_origin(x, y, W, H, &cx, &cy)) {
      ri.valid = 1;
      ri.base = (long long)(cy - ry) * W + (cx - rx);
      ri.feat[0] = (float)(2.0 * (x - (double)cx));
      ri.feat[1] = (float)(2.0 * (y - (double)cy));
      ri.feat[2] = (float)(i0 * sf.inv_i0ref_d);
    }
  } else {
    const double z = dummy[2 * stride + d];
    const double fx = floor(x + 0.5), fy = floor(y + 0.5), fz = floor(z + 0.5);
    if (fx - rx >= 0.0 && fx + rx <= (double)(W - 1) && fy - ry >= 0.0 && fy + ry <= (double)(H - 1) &&
        fz - rz >= 0.0 && fz + rz <= (double)(D - 1)) {
      const int cx = (int)fx, cy = (int)fy, cz = (int)fz;
      ri.valid = 1;
      ri.base = ((long long)(cz - rz) * H + (cy - ry)) * W + (cx - rx);
      ri.feat[0] = (float)(2.0 * (x - fx));
      ri.feat[1] = (float)(2.0 * (y - fy));
      ri.feat[2] = (float)(2.0 * (z - fz));
      ri.feat[3] = (float)(i0 * sf.inv_i0ref_d);
    }
  }
  return ri;
}

// offset of patch value f from the patch's first voxel
__device__ __forceinline__ int sur_poff(const SurGeom& g, int f, int W, int H) {
  if (f >= g.npix) return 0;
  const int pxy = g.px * g.py;
  return ((f / pxy) * H + (f % pxy) / g.px) * W + (f % g.px);
}

__device__ __forceinline__ float sur_input(const SurGeom& g, const float* __restrict__ img, const SurRowInfo& ri,
                                           int f, int poff_f, const SurFeat& sf) {
  if (f < g.npix) return (__ldg(img + ri.base + poff_f) - sf.bg) * sf.inv_i0ref;
  const int j = f - g.npix;
  if (j < g.nfeat - 1) return ri.feat[j];
  if (j == g.nfeat - 1) return sf.sig_feat;
  return 0.0f;
}

// index of the window term of the window whose first voxel is at base (its centre voxel)
__device__ __forceinline__ long long sur_tindex(const SurGeom& g, long long base, int W, int H) {
  return base + ((long long)(g.pz >> 1) * H + (g.py >> 1)) * W + (g.px >> 1);
}

// ---------------------------------------------------------------------------
// Window term T(cx, cy) = sum over the 21 x 21 window of
// (z - z log z + log(bg) z) - 441 bg, for every window inside the image
// (NaN elsewhere).  Per-pixel terms in FP32, window sums in double-float
// (pairs of FP32 with error-free additions: GB300's FP64 pipe would make this
// pass cost more than the network), stored rounded to FP32 (relative error
// 2^-24, 1e-4 nats for |T| ~ 1e3).  One block per 32 x 32 tile of window
// centres, the (32 + 20)^2 input pixels staged in shared memory, a
// horizontal then a vertical pass of 21-wide sums.
// ---------------------------------------------------------------------------
constexpr int WT_TILE = 32;
constexpr int WT_IN = WT_TILE + 2 * SUR_R;  // 52

__global__ void __launch_bounds__(256)
k_sur_window(const float* __restrict__ img, int W, int H, float log_bg, df pbg, float* __restrict__ T) {
  __shared__ float s_v[WT_IN][WT_IN];
  __shared__ float s_hh[WT_IN][WT_TILE], s_hl[WT_IN][WT_TILE];
  const int x0 = blockIdx.x * WT_TILE, y0 = blockIdx.y * WT_TILE;
  for (int i = threadIdx.x; i < WT_IN * WT_IN; i += blockDim.x) {
    const int yy = y0 - SUR_R + i / WT_IN, xx = x0 - SUR_R + i % WT_IN;
    float v = 0.0f;
    if (xx >= 0 && xx < W && yy >= 0 && yy < H) {
      const float z = img[(long long)yy * W + xx];
      v = (z > 0.0f ? z - z * logf(z) : 0.0f) + log_bg * z;
    }
    s_v[i / WT_IN][i % WT_IN] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < WT_IN * WT_TILE; i += blockDim.x) {
    const int r = i / WT_TILE, c = i % WT_TILE;
    df a{0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 2 * SUR_R + 1; ++k) a = df_add_f(a, s_v[r][c + k]);
    s_hh[r][c] = a.hi;
    s_hl[r][c] = a.lo;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < WT_TILE * WT_TILE; i += blockDim.x) {
    const int r = i / WT_TILE, c = i % WT_TILE;
    const int x = x0 + c, y = y0 + r;
    if (x >= W || y >= H) continue;
    df a{0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 2 * SUR_R + 1; ++k) a = df_add(a, df{s_hh[r + k][c], s_hl[r + k][c]});
    a = df_add(a, df{-pbg.hi, -pbg.lo});
    const bool inside = x >= SUR_R && x + SUR_R <= W - 1 && y >= SUR_R && y + SUR_R <= H - 1;
    T[(long long)y * W + x] = inside ? a.hi + a.lo : __int_as_float(0x7fc00000);
  }
}


// 3D window term: T(cx, cy, cz) = sum over the px x py x pz window of
// (z - z log z + log(bg) z) - npix bg, for every window inside the volume (NaN
// elsewhere).  Three separable passes (x, y, z), each summing in double-float
// (pairs of FP32); the per-voxel term is formed in the x pass.
__global__ void k_sur_win3_x(const float* __restrict__ vol, int W, int H, int D, int rx, float log_bg,
                             float* __restrict__ ah, float* __restrict__ al) {
  const long long n = (long long)W * H * D;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % W);
    df acc{0.0f, 0.0f};
    for (int k = -rx; k <= rx; ++k) {
      const int xx = x + k;
      if (xx < 0 || xx >= W) continue;
      const float z = vol[i + k];
      acc = df_add_f(acc, (z > 0.0f ? z - z * logf(z) : 0.0f) + log_bg * z);
    }
    ah[i] = acc.hi;
    al[i] = acc.lo;
  }
}

// one separable pass along y (stride W, extent H) or z (stride W H, extent D)
__global__ void k_sur_win3_pass(const float* __restrict__ ih, const float* __restrict__ il, int W, int H, int D,
                                int axis, int r, float* __restrict__ oh, float* __restrict__ ol) {
  const long long n = (long long)W * H * D;
  const long long stride = axis == 1 ? (long long)W : (long long)W * H;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = axis == 1 ? (int)((i / W) % H) : (int)(i / ((long long)W * H));
    const int ext = axis == 1 ? H : D;
    df acc{0.0f, 0.0f};
    for (int k = -r; k <= r; ++k) {
      const int cc = c + k;
      if (cc < 0 || cc >= ext) continue;
      acc = df_add(acc, df{ih[i + k * stride], il[i + k * stride]});
    }
    oh[i] = acc.hi;
    ol[i] = acc.lo;
  }
}

__global__ void k_sur_win3_final(const float* __restrict__ ih, const float* __restrict__ il, int W, int H, int D,
                                 int rx, int ry, int rz, df pbg, float* __restrict__ T) {
  const long long n = (long long)W * H * D;
  const long long plane = (long long)W * H;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % W), y = (int)((i / W) % H), z = (int)(i / plane);
    df acc{0.0f, 0.0f};
    for (int k = -rz; k <= rz; ++k) {
      const int zz = z + k;
      if (zz < 0 || zz >= D) continue;
      acc = df_add(acc, df{ih[i + k * plane], il[i + k * plane]});
    }
    acc = df_add(acc, df{-pbg.hi, -pbg.lo});
    const bool inside = x >= rx && x + rx <= W - 1 && y >= ry && y + ry <= H - 1 && z >= rz && z + rz <= D - 1;
    T[i] = inside ? acc.hi + acc.lo : __int_as_float(0x7fc00000);
  }
}

// ---------------------------------------------------------------------------
// Parameters: random initial values and bf16 copies.
// ---------------------------------------------------------------------------
__global__ void k_sur_init(float* __restrict__ P, unsigned long long seed, SurGeom gm) {
  const unsigned long long s0 = splitmix64(seed);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < gm.ndev; i += (long long)gridDim.x * blockDim.x) {
    const float u = (float)(splitmix64(s0 + (unsigned long long)i) >> 40) * (1.0f / 16777216.0f) * 2.0f - 1.0f;
    float v = 0.0f;
    if (i < gm.off_b1) {
      if ((int)(i % gm.k1) < gm.nin) v = u * sqrtf(3.0f / gm.nin);
    } else if (i >= gm.off_w2 && i < gm.off_b2) {
      v = u * sqrtf(3.0f / SUR_HID);
    } else if (i >= gm.off_w3 && i < gm.off_b3) {
      v = u * sqrtf(3.0f / SUR_HID);
    }
    P[i] = v;
  }
}

__global__ void k_sur_tobf16(const float* __restrict__ P, __nv_bfloat16* __restrict__ W1b,
                             __nv_bfloat16* __restrict__ W2b, SurGeom gm) {
  const long long n1 = (long long)SUR_HID * gm.k1, n2 = (long long)SUR_HID * SUR_HID;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2; i += (long long)gridDim.x * blockDim.x) {
    if (i < n1)
      W1b[i] = __float2bfloat16_rn(P[gm.off_w1 + i]);
    else
      W2b[i - n1] = __float2bfloat16_rn(P[gm.off_w2 + i - n1]);
  }
}

// ---------------------------------------------------------------------------
// Dataset rows.  Appending is deterministic: a first pass counts the
// non-clipped states per block of 256, a second places each block's rows
// after those of the earlier blocks, in state order.
// ---------------------------------------------------------------------------
constexpr int ADD_THREADS = 256;

__global__ void __launch_bounds__(ADD_THREADS)
k_sur_add_count(SurGeom gm, const double* __restrict__ dummy, long long stride, long long n, int W, int H, int D,
                unsigned* __restrict__ blk_cnt, const unsigned long long* __restrict__ count,
                unsigned long long* __restrict__ base) {
  const long long d = (long long)blockIdx.x * ADD_THREADS + threadIdx.x;
  int ok = 0;
  if (d < n) ok = sur_row_info(gm, dummy, stride, d, W, H, D, SurFeat{0.f, 0.f, 0.f, 0.0}).valid;
  const int c = __syncthreads_count(ok);
  if (threadIdx.x == 0) {
    blk_cnt[blockIdx.x] = (unsigned)c;
    if (blockIdx.x == 0) *base = *count;
  }
}

__global__ void __launch_bounds__(ADD_THREADS)
k_sur_add_write(SurGeom gm, const double* __restrict__ dummy, long long stride, long long n,
                const double* __restrict__ ll, double label_floor, const float* __restrict__ T,
                const float* __restrict__ img, int W, int H, int D, SurFeat sf, const unsigned* __restrict__ blk_cnt,
                const unsigned long long* __restrict__ base, unsigned long long* __restrict__ count,
                unsigned* __restrict__ done, long long capacity, __nv_bfloat16* __restrict__ X,
                float* __restrict__ y, uint8_t* __restrict__ cens) {
  __shared__ unsigned long long s_off;
  __shared__ SurRowInfo s_ri[ADD_THREADS];
  __shared__ long long s_src[ADD_THREADS];
  __shared__ unsigned s_wsum[ADD_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // rows of the earlier blocks
  unsigned long long acc = 0;
  for (unsigned j = tid; j < blockIdx.x; j += ADD_THREADS) acc += blk_cnt[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (tid == 0) s_off = 0;
  __syncthreads();
  if (lane == 0) atomicAdd(&s_off, acc);
  // this block's states: validity and the exclusive rank among the valid ones
  const long long d = (long long)blockIdx.x * ADD_THREADS + tid;
  SurRowInfo ri{0, {0.f, 0.f, 0.f, 0.f}, 0};
  if (d < n) ri = sur_row_info(gm, dummy, stride, d, W, H, D, sf);
  const unsigned bal = __ballot_sync(0xffffffffu, ri.valid != 0);
  if (lane == 0) s_wsum[warp] = __popc(bal);
  __syncthreads();
  unsigned before = 0;
  for (int w = 0; w < warp; ++w) before += s_wsum[w];
  const unsigned rank = before + __popc(bal & ((1u << lane) - 1u));
  if (ri.valid) {
    s_ri[rank] = ri;
    s_src[rank] = d;
  }
  unsigned total = 0;
  for (int w = 0; w < ADD_THREADS / 32; ++w) total += s_wsum[w];
  __syncthreads();
  const unsigned long long off = *base + s_off;
  // one warp per row: k1 inputs, k1 / 32 per lane
  for (int r = warp; r < (int)total; r += ADD_THREADS / 32) {
    const unsigned long long row = off + (unsigned long long)r;
    if (row >= (unsigned long long)capacity) break;
    const SurRowInfo q = s_ri[r];
    for (int f = lane; f < gm.k1; f += 32)
      X[row * gm.k1 + f] = __float2bfloat16_rn(sur_input(gm, img, q, f, sur_poff(gm, f, W, H), sf));
    if (lane == 0) {
      const double v = ll[s_src[r]];
      const bool below = v < label_floor;
      y[row] = (float)((below ? label_floor : v) - (double)T[sur_tindex(gm, q.base, W, H)]);
      cens[row] = below ? 1 : 0;
    }
  }
  // the last block publishes the new row count
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      unsigned long long sum = 0;
      for (unsigned j = 0; j < gridDim.x; ++j) sum += ((volatile const unsigned*)blk_cnt)[j];
      unsigned long long c = *base + sum;
      *count = c < (unsigned long long)capacity ? c : (unsigned long long)capacity;
      *done = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// Label normalisation: sums over rows for the mean and the variance.
// ---------------------------------------------------------------------------
__global__ void k_sur_sums(const float* __restrict__ y, long long begin, long long end, double center,
                           double* __restrict__ acc) {
  double s = 0.0, s2 = 0.0;
  for (long long i = begin + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < end;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = (double)y[i] - center;
    s += v;
    s2 += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, s);
    atomicAdd(acc + 1, s2);
  }
}

// ---------------------------------------------------------------------------
// Training: minibatch gather, output head, Adam.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long sur_batch_row(long long begin, long long range, unsigned long long seed,
                                                   long long step, int i, int bt) {
  if (seed == 0ull) return begin + (long long)(((unsigned long long)step * (unsigned long long)bt + (unsigned)i) %
                                               (unsigned long long)range);
  const unsigned long long h =
      splitmix64(splitmix64(seed) + (((unsigned long long)step << 32) | (unsigned long long)(unsigned)i));
  return begin + (long long)(h % (unsigned long long)range);
}

// one warp per minibatch row: k1 bf16 inputs (k1 / 8 x 16 bytes) and the normalised label
__global__ void k_sur_gather(const __nv_bfloat16* __restrict__ X, const float* __restrict__ y,
                             const uint8_t* __restrict__ cens, long long begin, long long range,
                             unsigned long long seed, long long step, int bt, const double* __restrict__ norm,
                             __nv_bfloat16* __restrict__ Xb, float* __restrict__ yb, uint8_t* __restrict__ cb, int k1) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= bt) return;
  const long long r = sur_batch_row(begin, range, seed, step, i, bt);
  const uint4* src = reinterpret_cast<const uint4*>(X + r * k1);
  uint4* dst = reinterpret_cast<uint4*>(Xb + (long long)i * k1);
  for (int j = lane; j < k1 / 8; j += 32) dst[j] = src[j];
  if (lane == 0) {
    yb[i] = (float)(((double)y[r] - norm[0]) / norm[1]);
    cb[i] = cens[r];
  }
}

// Output layer and its backward pass, one warp per row (8 hidden units per
// lane): a2 = silu(z2), out = w3 . a2 + b3, d = out - t (0 for a censored row
// with out <= t), loss += d^2 / bt, g = 2 d / bt; G2 = bf16(g w3 silu'(z2));
// gradients of w3, b2, b3 summed per block, then added to the global
// gradient.
constexpr int HEAD_THREADS = 256;

__global__ void __launch_bounds__(HEAD_THREADS)
k_sur_head(const float* __restrict__ Z2, const float* __restrict__ yb, const uint8_t* __restrict__ cb, int bt,
           const float* __restrict__ P,
           float* __restrict__ G, __nv_bfloat16* __restrict__ G2, float* __restrict__ loss, SurGeom gm) {
  __shared__ float s_w3[SUR_HID], s_db2[SUR_HID];
  __shared__ float s_misc[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = tid; j < SUR_HID; j += HEAD_THREADS) {
    s_w3[j] = 0.0f;
    s_db2[j] = 0.0f;
  }
  if (tid < 2) s_misc[tid] = 0.0f;
  __syncthreads();
  const float* w3 = P + gm.off_w3;
  const float b3 = P[gm.off_b3];
  float wl[8], dw3[8], db2[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    wl[k] = w3[lane * 8 + k];
    dw3[k] = 0.0f;
    db2[k] = 0.0f;
  }
  float db3 = 0.0f, lsum = 0.0f;
  const float inv_bt = 1.0f / (float)bt;
  for (int i = blockIdx.x * (HEAD_THREADS / 32) + warp; i < bt; i += gridDim.x * (HEAD_THREADS / 32)) {
    const float4* zp = reinterpret_cast<const float4*>(Z2 + (long long)i * SUR_HID + lane * 8);
    const float4 za = zp[0], zb = zp[1];
    const float z[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
    float a[8], part = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      a[k] = silu_f(z[k]);
      part = fmaf(a[k], wl[k], part);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    float d = part + b3 - yb[i];
    if (cb[i] && d < 0.0f) d = 0.0f;
    const float g = 2.0f * d * inv_bt;
    lsum += d * d * inv_bt;
    db3 += g;
    float gz[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      dw3[k] = fmaf(g, a[k], dw3[k]);
      gz[k] = g * wl[k] * silu_grad_f(z[k]);
      db2[k] += gz[k];
    }
    *reinterpret_cast<uint4*>(G2 + (long long)i * SUR_HID + lane * 8) = pack_bf16x8(gz);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    atomicAdd(&s_w3[lane * 8 + k], dw3[k]);
    atomicAdd(&s_db2[lane * 8 + k], db2[k]);
  }
  if (lane == 0) {
    atomicAdd(&s_misc[0], db3);
    atomicAdd(&s_misc[1], lsum);
  }
  __syncthreads();
  for (int j = tid; j < SUR_HID; j += HEAD_THREADS) {
    atomicAdd(G + gm.off_w3 + j, s_w3[j]);
    atomicAdd(G + gm.off_b2 + j, s_db2[j]);
  }
  if (tid == 0) {
    atomicAdd(G + gm.off_b3, s_misc[0]);
    if (loss) atomicAdd(loss, s_misc[1]);
  }
}

// Adam with bias-corrected moments (c1 = 1 / (1 - beta1^t), c2 = 1 / (1 -
// beta2^t)); zeroes the gradient for the next minibatch and refreshes the
// bf16 weight copies.
__global__ void k_sur_adam(float* __restrict__ P, float* __restrict__ G, float* __restrict__ Mo,
                           float* __restrict__ V, float lr, float c1, float c2, __nv_bfloat16* __restrict__ W1b,
                           __nv_bfloat16* __restrict__ W2b, SurGeom gm) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < gm.ndev; i += (long long)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * Mo[i] + (1.0f - b1) * g;
    const float v = b2 * V[i] + (1.0f - b2) * g * g;
    Mo[i] = m;
    V[i] = v;
    const float p = P[i] - lr * (m * c1) / (sqrtf(v * c2) + eps);
    P[i] = p;
    G[i] = 0.0f;
    if (i < gm.off_b1)
      W1b[i] = __float2bfloat16_rn(p);
    else if (i >= gm.off_w2 && i < gm.off_b2)
      W2b[i - gm.off_w2] = __float2bfloat16_rn(p);
  }
}

// ---------------------------------------------------------------------------
// Fused inference.  Per tile of 128 states the inputs are built from the
// image straight into the shared-memory operand layout; layer 1 (K = k1:
// 448 in 2D, seven chunks of 64; 896 in 3D) and layer 2 (K = 256, four chunks, the bf16
// activations of layer 1 kept in shared memory) accumulate in the same 256
// TMEM columns, and the output layer runs in FP32 on the TMEM lanes.
//
// The weight chunks (32 KB each, k1 / 64 + 4 of them) are stored pre-arranged in the
// swizzled shared-memory layout, so one thread fetches a chunk with a single
// bulk asynchronous copy completing on an mbarrier.  Input and weight
// buffers are doubled: the copy and the input build of chunk q overlap the
// MMAs of chunk q - 1.  Eight warps: all build inputs; for the epilogues the
// warps w and w + 4 share TMEM lanes 32 (w mod 4) .. + 31 and split the 256
// columns in halves.
// ---------------------------------------------------------------------------
constexpr int SI_THREADS = 256;
constexpr int SI_CHUNKS_MAX = SUR_K1_MAX / MM_K + SUR_HID / MM_K;  // 14 + 4 (3D)
constexpr int SI_X = 128 * MM_K * 2;      // 16 KB: one input chunk
constexpr int SI_W = SUR_HID * MM_K * 2;  // 32 KB: one weight chunk
constexpr int SI_A = 128 * SUR_HID * 2;   // 64 KB: layer-1 activations (four chunks)
constexpr int SI_SMEM = 2 * SI_X + 2 * SI_W + SI_A + SUR_K1_MAX * 4 + 128 * (int)sizeof(SurRowInfo) +
                        2 * 128 * 4 + 64;
enum { SRC_STATES = 0, SRC_ROWS = 1 };

struct SurNet {
  const uint8_t* Wsw;   // k1 / 64 + 4 weight chunks in the shared-memory layout
  const float* P;       // FP32 parameters (biases, output layer)
  const double* norm;   // label mean and scale
};

struct SurInfer {
  SurNet net;
  SurGeom gm;
  const double* dummy;
  long long stride;
  const __nv_bfloat16* rows;
  long long n;
  const unsigned* n_dev;  // when set, the count is *n_dev
  const float* img;
  int W, H, D;
  SurFeat sf;
  const float* T;                 // window terms of img (states), or null (rows: label units)
  double* out;
  int nan_clipped;                // write NaN for clipped states
  unsigned long long* max_ll;     // ordered maximum of the written predictions, or null
  unsigned* bad;                  // set when a prediction is not finite (or null)
  unsigned* err;
};

// weight chunk q (W1 for q < k1 / 64, W2 after) rearranged into the shared-memory layout
__global__ void k_sur_pack(const __nv_bfloat16* __restrict__ W1b, const __nv_bfloat16* __restrict__ W2b,
                           uint8_t* __restrict__ Wsw, int k1) {
  const int c1 = k1 / MM_K;
  const int total = (c1 + SUR_HID / MM_K) * SUR_HID * 8;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    const int q = g / (SUR_HID * 8), rem = g % (SUR_HID * 8);
    const int r = rem >> 3, kg = (rem & 7) * 8;
    const uint4 v = q < c1 ? *reinterpret_cast<const uint4*>(W1b + (long long)r * k1 + q * MM_K + kg)
                           : *reinterpret_cast<const uint4*>(W2b + (long long)r * SUR_HID + (q - c1) * MM_K + kg);
    *reinterpret_cast<uint4*>(Wsw + (long long)q * SI_W + mm_off(r, kg)) = v;
  }
}

__device__ __forceinline__ void bulk_load(uint8_t* dst, const uint8_t* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// 4 x 8 consecutive fp32 columns of this thread's TMEM lane, one wait
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
#pragma unroll
  for (int j = 0; j < 4; ++j)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[8 * j]), "=r"(r[8 * j + 1]), "=r"(r[8 * j + 2]), "=r"(r[8 * j + 3]), "=r"(r[8 * j + 4]),
          "=r"(r[8 * j + 5]), "=r"(r[8 * j + 6]), "=r"(r[8 * j + 7])
        : "r"(taddr + 8u * j)
        : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int SRC>
__global__ void __launch_bounds__(SI_THREADS, 1) k_sur_infer(SurInfer a) {
  extern __shared__ __align__(1024) uint8_t si_smem_raw[];
  uint8_t* sX = align1024(si_smem_raw);  // two input chunks
  uint8_t* sW = sX + 2 * SI_X;           // two weight chunks
  uint8_t* sA = sW + 2 * SI_W;           // layer-1 activations
  int* poff = reinterpret_cast<int*>(sA + SI_A);
  SurRowInfo* rowi = reinterpret_cast<SurRowInfo*>(poff + SUR_K1_MAX);
  float* part = reinterpret_cast<float*>(rowi + 128);  // [2][128] partial output sums
  uint64_t* bar_w = reinterpret_cast<uint64_t*>(part + 2 * 128);
  uint64_t* bar_m = bar_w + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar_m + 2);
  __shared__ double s_max[4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = 32 * (warp & 3) + lane;  // TMEM lane of this thread
  const int half = warp >> 2;               // column half of the epilogues
  const long long n = a.n_dev ? (long long)*a.n_dev : a.n;
  const long long ntiles = (n + 127) / 128;
  if ((long long)blockIdx.x >= ntiles) return;
  const SurGeom& gm = a.gm;
  const int c1 = gm.k1 / MM_K;              // input chunks of layer 1
  const int nchunks = c1 + SUR_HID / MM_K;  // and the four of layer 2
  for (int f = tid; f < gm.k1; f += SI_THREADS) poff[f] = sur_poff(gm, f, a.W, a.H);
  if (warp == 0) tc_alloc(tslot, SUR_HID);
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar_w[i], 1);
      mbar_init(&bar_m[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(half * 128);
  const uint32_t idesc = mm_idesc(128, SUR_HID);
  const float* b1 = a.net.P + gm.off_b1;
  const float* b2 = a.net.P + gm.off_b2;
  const float* w3 = a.net.P + gm.off_w3;
  const float b3 = a.net.P[gm.off_b3];
  const double mean = a.net.norm[0], scale = a.net.norm[1];
  uint32_t ph_w[2] = {0u, 0u}, ph_m[2] = {0u, 0u};
  bool out_w[2] = {false, false}, out_m[2] = {false, false};  // copy / MMA in flight on buffer b
  bool ok = true;
  double mymax = -INFINITY;
  unsigned q = 0;  // running chunk counter: buffer q & 1

  // bounded wait for the MMA last committed on buffer b (uniform over the block)
  auto wait_mma = [&](int b) {
    if (!out_m[b]) return;
    ok = ok && __syncthreads_and(tid != 0 || mbar_wait(&bar_m[b], ph_m[b])) != 0;
    ph_m[b] ^= 1u;
    out_m[b] = false;
    tc_fence_after();
  };

  for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const long long d = t * 128 + (tid & 127);
    if (tid < 128) {
      if (SRC == SRC_STATES) {
        SurRowInfo ri{0, {0.f, 0.f, 0.f, 0.f}, 0};
        if (d < n) ri = sur_row_info(gm, a.dummy, a.stride, d, a.W, a.H, a.D, a.sf);
        rowi[tid] = ri;
      } else {
        rowi[tid] = SurRowInfo{0, {0.f, 0.f, 0.f, 0.f}, d < n ? 1 : 0};
      }
    }
    __syncthreads();
    for (int c = 0; c < nchunks && ok; ++c, ++q) {
      const int b = q & 1;
      wait_mma(b);  // buffers b free again
      if (!ok) break;
      if (tid == 0) {
        bulk_load(sW + b * SI_W, a.net.Wsw + (long long)c * SI_W, SI_W, &bar_w[b]);
        out_w[b] = true;
      }
      if (c < c1) {
        // inputs of chunk c: 128 rows x 8 groups of 8, four groups per thread, loads first
        float v[4][8];
        uint4 u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int g = tid + j * SI_THREADS;
          const int r = g >> 3, kg = (g & 7) * 8;
          const SurRowInfo ri = rowi[r];
          if (SRC == SRC_ROWS) {
            u[j] = ri.valid ? __ldg(reinterpret_cast<const uint4*>(a.rows + (t * 128 + r) * gm.k1 + c * MM_K + kg))
                            : make_uint4(0u, 0u, 0u, 0u);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int f = c * MM_K + kg + i;
              v[j][i] = ri.valid ? sur_input(gm, a.img, ri, f, poff[f], a.sf) : 0.0f;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int g = tid + j * SI_THREADS;
          const int r = g >> 3, kg = (g & 7) * 8;
          if (SRC == SRC_STATES) u[j] = pack_bf16x8(v[j]);
          *reinterpret_cast<uint4*>(sX + b * SI_X + mm_off(r, kg)) = u[j];
        }
      } else if (c == c1) {
        // layer-1 epilogue: all layer-1 MMAs done (the other buffer's too), then bias, SiLU, bf16
        wait_mma(b ^ 1);
        if (!ok) break;
#pragma unroll 1
        for (int cc = 0; cc < 128; cc += 32) {
          float v[32];
          tc_ld32(taddr + (uint32_t)cc, v);
          const int col0 = half * 128 + cc;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float w[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) w[i] = silu_f(v[8 * j + i] + __ldg(b1 + col0 + 8 * j + i));
            const int col = col0 + 8 * j;
            *reinterpret_cast<uint4*>(sA + (col / MM_K) * SI_X + mm_off(row, col % MM_K)) = pack_bf16x8(w);
          }
        }
        tc_fence_before();
      }
      proxy_fence();
      __syncthreads();
      // weights of chunk c present
      ok = ok && __syncthreads_and(tid != 0 || mbar_wait(&bar_w[b], ph_w[b])) != 0;
      ph_w[b] ^= 1u;
      out_w[b] = false;
      if (!ok) break;
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = c < c1 ? smem_u32(sX + b * SI_X) : smem_u32(sA + (c - c1) * SI_X);
        tc_mma_chunk(tmem, a0, smem_u32(sW + b * SI_W), idesc, c == 0 || c == c1);
        tc_commit(&bar_m[b]);
      }
      out_m[b] = true;
    }
    if (!ok) break;
    wait_mma(0);
    wait_mma(1);
    if (!ok) break;
    // output layer in FP32: each half sums its 128 columns
    float acc = 0.0f;
#pragma unroll 1
    for (int cc = 0; cc < 128; cc += 32) {
      float v[32];
      tc_ld32(taddr + (uint32_t)cc, v);
      const int col0 = half * 128 + cc;
#pragma unroll
      for (int i = 0; i < 32; ++i) acc = fmaf(silu_f(v[i] + __ldg(b2 + col0 + i)), __ldg(w3 + col0 + i), acc);
    }
    part[half * 128 + row] = acc;
    tc_fence_before();
    __syncthreads();
    if (tid < 128) {
      const long long dd = t * 128 + tid;
      double ll = mean + scale * (double)(part[tid] + part[128 + tid] + b3);
      if (SRC == SRC_STATES && rowi[tid].valid) ll += (double)a.T[sur_tindex(gm, rowi[tid].base, a.W, a.H)];
      if (rowi[tid].valid) {
        if (!isfinite(ll) && a.bad) atomicOr(a.bad, 1u);
        a.out[dd] = ll;
        mymax = fmax(mymax, ll);
      } else if (a.nan_clipped && dd < n) {
        a.out[dd] = __longlong_as_double(0x7ff8000000000000ll);
      }
    }
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicOr(a.err, (unsigned)PCSIR_DERR_TIMEOUT);
    // let copies still in flight land before the block's shared memory goes away
    for (int b = 0; b < 2; ++b)
      if (out_w[b]) mbar_wait(&bar_w[b], ph_w[b]);
  }
  if (a.max_ll) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mymax = fmax(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    if (lane == 0 && warp < 4) s_max[warp] = mymax;
    __syncthreads();
    if (tid == 0) {
      double m = -INFINITY;
      for (int w = 0; w < 4; ++w) m = fmax(m, s_max[w]);
      if (m > -INFINITY) atomicMax(a.max_ll, ord_encode(m));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, SUR_HID);
}

// ---------------------------------------------------------------------------
// Held-out check of a surrogate-assisted step (one block).
// ---------------------------------------------------------------------------
constexpr int CHK_THREADS = 256;

__global__ void __launch_bounds__(CHK_THREADS)
k_sur_check(Control* __restrict__ ctl, const double* __restrict__ bin_ll, SurStats* __restrict__ st,
            const int* __restrict__ ho_bin, const double* __restrict__ ho_ll, int ho_cap, double window,
            double max_err) {
  __shared__ double s_mx[CHK_THREADS / 32], s_ss[CHK_THREADS / 32];
  __shared__ unsigned s_ns[CHK_THREADS / 32], s_nf[CHK_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned nho = min(st->n_ho, (unsigned)ho_cap);
  const unsigned long long me = ctl->max_ll;
  const double maxp = me == 0ull ? -INFINITY : ord_decode(me);
  double mx = 0.0, ss = 0.0;
  unsigned ns = 0, nf = 0;
  for (unsigned i = tid; i < nho; i += CHK_THREADS) {
    const double p = bin_ll[ho_bin[i]], e = ho_ll[i];
    const double err = fabs(p - e);
    if (isfinite(err)) {
      ss += err * err;
    } else {
      ++nf;
    }
    if (fmax(p, e) >= maxp - window) {
      ++ns;
      mx = fmax(mx, isnan(err) ? INFINITY : err);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    ns += __shfl_xor_sync(0xffffffffu, ns, o);
    nf += __shfl_xor_sync(0xffffffffu, nf, o);
  }
  if (lane == 0) {
    s_mx[warp] = mx;
    s_ss[warp] = ss;
    s_ns[warp] = ns;
    s_nf[warp] = nf;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < CHK_THREADS / 32; ++w) {
      mx = fmax(mx, s_mx[w]);
      ss += s_ss[w];
      ns += s_ns[w];
      nf += s_nf[w];
    }
    // s_*[0] already included through the thread's own registers (warp 0)
    st->max_err = mx;
    st->sum_sq = ss;
    st->n_sig = ns;
    st->n_nonfinite_err = nf;
    const bool fb = !(mx <= max_err) || nf > 0u || st->bad != 0u;
    st->fallback = fb ? 1u : 0u;
    if (fb) ctl->max_ll = 0ull;  // the exact pass recomputes the maximum
  }
}

cudaError_t prepare_surrogate() {
  static std::once_flag once;
  static cudaError_t status = cudaSuccess;
  std::call_once(once, [] {
    status = cudaFuncSetAttribute(k_sur_infer<SRC_STATES>, cudaFuncAttributeMaxDynamicSharedMemorySize, SI_SMEM + 1024);
    if (status == cudaSuccess)
      status = cudaFuncSetAttribute(k_sur_infer<SRC_ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, SI_SMEM + 1024);
    if (status == cudaSuccess) status = prepare_gemm();
  });
  return status;
}

}  // namespace pcsir

using namespace pcsir;

struct pcsir_surrogate {
  pcsir_surrogate_config cfg{};
  int device = 0;
  int num_sms = 0;
  float *P = nullptr, *G = nullptr, *Mo = nullptr, *V = nullptr;
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr;
  SurGeom gm{};            // input geometry (2D or 3D patch)
  uint8_t* Wsw = nullptr;  // (k1 / 64 + 4) x 32 KB, inference layout
  double* norm = nullptr;  // device: label mean, scale
  double host_mean = 0.0, host_scale = 1.0;
  __nv_bfloat16* X = nullptr;
  float* y = nullptr;
  uint8_t* cens = nullptr;
  uint8_t* cb = nullptr;
  float* T = nullptr;  // window terms of the current image (max_pixels)
  float* wbuf = nullptr;  // 3D: scratch of the separable window passes (4 x max_pixels)
  unsigned long long* count = nullptr;
  unsigned long long* add_base = nullptr;
  unsigned* add_cnt = nullptr;
  unsigned* add_done = nullptr;
  long long add_max_blocks = 0;
  __nv_bfloat16 *Xb = nullptr, *A1 = nullptr, *G2 = nullptr, *G1 = nullptr;
  float *yb = nullptr, *Z1 = nullptr, *Z2 = nullptr, *loss_scratch = nullptr;
  double* fit_acc = nullptr;
  unsigned* err = nullptr;
  long long adam_t = 0;
  std::vector<void*> allocs;
  std::string errmsg = "no error";
};

namespace {

pcsir_status sfail(pcsir_surrogate* s, pcsir_status st, const std::string& msg) {
  if (s) s->errmsg = msg;
  return st;
}
pcsir_status scuda(pcsir_surrogate* s, cudaError_t e, const char* what) {
  cudaGetLastError();
  return sfail(s, PCSIR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
bool salloc(pcsir_surrogate* s, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  s->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return true;
}

void sfree(pcsir_surrogate* s) {
  for (void* p : s->allocs) cudaFree(p);
  s->allocs.clear();
}

int grid_for(long long n, int threads, int num_sms) {
  const long long want = (n + threads - 1) / threads;
  return (int)std::max<long long>(1, std::min<long long>(want, (long long)num_sms * 8));
}

SurFeat make_feat(const pcsir_surrogate* s, double bg, double sigma) {
  SurFeat f;
  f.bg = (float)bg;
  f.inv_i0ref = (float)(1.0 / s->cfg.i0_ref);
  f.inv_i0ref_d = 1.0 / s->cfg.i0_ref;
  f.sig_feat = (float)(sigma / s->cfg.sigma_ref);
  return f;
}

SurNet net_of(const pcsir_surrogate* s) { return SurNet{s->Wsw, s->P, s->norm}; }

// inference copy of the weights in the shared-memory layout (after any change of W1b / W2b)
cudaError_t pack_weights(const pcsir_surrogate* s, cudaStream_t st) {
  k_sur_pack<<<2 * s->num_sms, 256, 0, st>>>(s->W1b, s->W2b, s->Wsw, s->gm.k1);
  return cudaGetLastError();
}

cudaError_t launch_window(const pcsir_surrogate* s, const float* img, int W, int H, int D, double bg,
                          cudaStream_t st) {
  if ((long long)W * H * D > s->cfg.max_pixels) return cudaErrorInvalidValue;
  const double pbg = (double)s->gm.npix * bg;
  const df pbg_df{(float)pbg, (float)(pbg - (double)(float)pbg)};
  if (s->gm.dim == 2) {
    dim3 grid((W + WT_TILE - 1) / WT_TILE, (H + WT_TILE - 1) / WT_TILE);
    k_sur_window<<<grid, 256, 0, st>>>(img, W, H, (float)std::log(bg), pbg_df, s->T);
    return cudaGetLastError();
  }
  const long long n = (long long)W * H * D;
  const int grid = grid_for(n, 256, s->num_sms);
  float* ah = s->wbuf;
  float* al = ah + s->cfg.max_pixels;
  float* bh = al + s->cfg.max_pixels;
  float* bl = bh + s->cfg.max_pixels;
  k_sur_win3_x<<<grid, 256, 0, st>>>(img, W, H, D, s->gm.px >> 1, (float)std::log(bg), ah, al);
  k_sur_win3_pass<<<grid, 256, 0, st>>>(ah, al, W, H, D, 1, s->gm.py >> 1, bh, bl);
  k_sur_win3_final<<<grid, 256, 0, st>>>(bh, bl, W, H, D, s->gm.px >> 1, s->gm.py >> 1, s->gm.pz >> 1, pbg_df, s->T);
  return cudaGetLastError();
}

cudaError_t launch_infer(const pcsir_surrogate* s, const SurInfer& a, int src, long long ntiles_max,
                         cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>(ntiles_max, (long long)s->num_sms));
  if (src == SRC_STATES)
    k_sur_infer<SRC_STATES><<<grid, SI_THREADS, SI_SMEM + 1024, st>>>(a);
  else
    k_sur_infer<SRC_ROWS><<<grid, SI_THREADS, SI_SMEM + 1024, st>>>(a);
  return cudaGetLastError();
}

// forward and backward of one minibatch already gathered into Xb / yb (bt rows);
// the gradient accumulates into s->G (which must be zero)
cudaError_t fwd_bwd(pcsir_surrogate* s, int bt, float* loss, cudaStream_t st) {
  const int sms = s->num_sms;
  const int mt = (bt + 127) / 128;
  const int nt_act = mt >= sms / 2 ? 256 : 64;  // narrower column tiles when the rows alone fill few SMs
  GemmArgs g{};
  g.err = s->err;
  // layer 1: Z1 = Xb W1^T + b1, A1 = silu(Z1)
  g.A = s->Xb; g.sam = s->gm.k1; g.sak = 1;
  g.B = s->W1b; g.sbn = s->gm.k1; g.sbk = 1;
  g.C = s->Z1; g.ldc = SUR_HID;
  g.M = bt; g.N = SUR_HID; g.K = s->gm.k1;
  g.epi = EPI_ACT; g.bias = s->P + s->gm.off_b1; g.act = s->A1; g.ld_act = SUR_HID;
  cudaError_t e = launch_gemm(g, st, nt_act, 1);
  if (e != cudaSuccess) return e;
  // layer 2: Z2 = A1 W2^T + b2
  g.A = s->A1; g.sam = SUR_HID; g.sak = 1;
  g.B = s->W2b; g.sbn = SUR_HID; g.sbk = 1;
  g.C = s->Z2; g.K = SUR_HID;
  g.bias = s->P + s->gm.off_b2; g.act = nullptr;
  if ((e = launch_gemm(g, st, nt_act, 1)) != cudaSuccess) return e;
  // output layer, loss, G2 and the gradients of w3, b2, b3
  k_sur_head<<<std::min(mt * 4, sms * 2), HEAD_THREADS, 0, st>>>(s->Z2, s->yb, s->cb, bt, s->P, s->G, s->G2, loss,
                                                                   s->gm);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int kchunks = (bt + MM_K - 1) / MM_K;
  // dW2 = G2^T A1 (both read with rows contiguous), split K
  GemmArgs w{};
  w.err = s->err;
  w.A = s->G2; w.sam = 1; w.sak = SUR_HID;
  w.B = s->A1; w.sbn = 1; w.sbk = SUR_HID;
  w.C = s->G + s->gm.off_w2; w.ldc = SUR_HID;
  w.M = SUR_HID; w.N = SUR_HID; w.K = bt;
  w.epi = EPI_ATOMIC;
  int splits = std::max(1, std::min(kchunks, sms / 2));
  if ((e = launch_gemm(w, st, 256, splits)) != cudaSuccess) return e;
  // G1 = (G2 W2) * silu'(Z1), db1 = column sums
  GemmArgs b{};
  b.err = s->err;
  b.A = s->G2; b.sam = SUR_HID; b.sak = 1;
  b.B = s->W2b; b.sbn = 1; b.sbk = SUR_HID;
  b.M = bt; b.N = SUR_HID; b.K = SUR_HID;
  b.epi = EPI_DACT; b.pre = s->Z1; b.ld_pre = SUR_HID; b.act = s->G1; b.ld_act = SUR_HID;
  b.colsum = s->G + s->gm.off_b1;
  if ((e = launch_gemm(b, st, nt_act, 1)) != cudaSuccess) return e;
  // dW1 = G1^T Xb, split K
  w.A = s->G1; w.sam = 1; w.sak = SUR_HID;
  w.B = s->Xb; w.sbn = 1; w.sbk = s->gm.k1;
  w.C = s->G + s->gm.off_w1; w.ldc = s->gm.k1;
  w.M = SUR_HID; w.N = s->gm.k1; w.K = bt;
  splits = std::max(1, std::min(kchunks, sms / 4));
  return launch_gemm(w, st, 256, splits);
}

}  // namespace

namespace pcsir {

int64_t sur_max_pixels(const pcsir_surrogate* s) { return s->cfg.max_pixels; }
int sur_dim(const pcsir_surrogate* s) { return s->gm.dim; }

cudaError_t launch_sur_step3(const SurStep& sp, const StepBuffers& b, double bg, double sigma_xy, const float* vol,
                             int W, int H, int D, cudaStream_t st) {
  const pcsir_surrogate* s = sp.sur;
  SurInfer a{};
  a.net = net_of(s);
  a.gm = s->gm;
  a.dummy = b.dummy;
  a.stride = b.bin_stride;
  a.n_dev = &b.ctl->nocc;
  a.img = vol;
  a.W = W;
  a.H = H;
  a.D = D;
  a.sf = make_feat(s, bg, sigma_xy);
  a.T = s->T;
  a.out = b.bin_ll;
  a.nan_clipped = 0;
  a.max_ll = &b.ctl->max_ll;
  a.bad = &sp.stats->bad;
  a.err = &b.ctl->err;
  cudaError_t e = launch_window(s, vol, W, H, D, bg, st);
  if (e != cudaSuccess) return e;
  e = launch_infer(s, a, SRC_STATES, (long long)s->num_sms, st);
  if (e != cudaSuccess) return e;
  k_sur_check<<<1, CHK_THREADS, 0, st>>>(b.ctl, b.bin_ll, sp.stats, sp.ho_bin, sp.ho_ll, sp.ho_cap, sp.window,
                                         sp.max_err);
  return cudaGetLastError();
}
void sur_refs(const pcsir_surrogate* s, double* i0_ref, double* sigma_ref) {
  *i0_ref = s->cfg.i0_ref;
  *sigma_ref = s->cfg.sigma_ref;
}

cudaError_t launch_sur_step(const SurStep& sp, const StepBuffers& b, const ModelParams& m, const float* img, int W,
                            int H, cudaStream_t st) {
  const pcsir_surrogate* s = sp.sur;
  SurInfer a{};
  a.net = net_of(s);
  a.gm = s->gm;
  a.D = 1;
  a.dummy = b.dummy;
  a.stride = b.bin_stride;
  a.n_dev = &b.ctl->nocc;
  a.img = img;
  a.W = W;
  a.H = H;
  a.sf = make_feat(s, m.bg, m.sigma);
  a.T = s->T;
  a.out = b.bin_ll;
  a.nan_clipped = 0;
  a.max_ll = &b.ctl->max_ll;
  a.bad = &sp.stats->bad;
  a.err = &b.ctl->err;
  cudaError_t e = launch_window(s, img, W, H, 1, m.bg, st);
  if (e != cudaSuccess) return e;
  e = launch_infer(s, a, SRC_STATES, (long long)s->num_sms, st);
  if (e != cudaSuccess) return e;
  k_sur_check<<<1, CHK_THREADS, 0, st>>>(b.ctl, b.bin_ll, sp.stats, sp.ho_bin, sp.ho_ll, sp.ho_cap, sp.window,
                                         sp.max_err);
  return cudaGetLastError();
}

}  // namespace pcsir

extern "C" {

const char* pcsir_surrogate_last_error(pcsir_surrogate* s) { return s ? s->errmsg.c_str() : "NULL surrogate"; }

pcsir_status pcsir_surrogate_create(const pcsir_surrogate_config* cfg, pcsir_surrogate** out) {
  if (!out) return PCSIR_EINVAL;
  *out = nullptr;
  if (!cfg || cfg->capacity < 1 || cfg->batch < 128 || cfg->batch > 65536 || (cfg->batch % 128) != 0 ||
      (cfg->geometry != 0 && cfg->geometry != 2 && cfg->geometry != 3) || !(cfg->i0_ref > 0.0) || !(cfg->sigma_ref > 0.0) || !std::isfinite(cfg->i0_ref) ||
      !std::isfinite(cfg->sigma_ref) || cfg->max_pixels < 1)
    return PCSIR_EINVAL;
  if (cfg->capacity > (int64_t(1) << 34)) return PCSIR_ERANGE;
  pcsir_surrogate* s = new (std::nothrow) pcsir_surrogate();
  if (!s) return PCSIR_ENOMEM;
  s->cfg = *cfg;
  s->gm = make_geom(cfg->geometry == 3 ? 3 : 2);
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
  if (e == cudaSuccess) e = prepare_surrogate();
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return PCSIR_ECUDA;
  }
  const size_t bt = (size_t)cfg->batch;
  const size_t cap = (size_t)cfg->capacity;
  s->add_max_blocks = 1 << 12;  // up to 2^20 states per add call
  bool ok = salloc(s, &s->P, s->gm.ndev) && salloc(s, &s->G, s->gm.ndev) && salloc(s, &s->Mo, s->gm.ndev) && salloc(s, &s->V, s->gm.ndev) &&
            salloc(s, &s->W1b, (size_t)SUR_HID * s->gm.k1) && salloc(s, &s->W2b, (size_t)SUR_HID * SUR_HID) &&
            salloc(s, &s->Wsw, (size_t)(s->gm.k1 / MM_K + SUR_HID / MM_K) * SI_W) &&
            salloc(s, &s->norm, 2) && salloc(s, &s->X, cap * s->gm.k1) && salloc(s, &s->y, cap) && salloc(s, &s->cens, cap) &&
            salloc(s, &s->cb, bt) &&
            salloc(s, &s->count, 1) && salloc(s, &s->add_base, 1) && salloc(s, &s->add_cnt, (size_t)s->add_max_blocks) &&
            salloc(s, &s->add_done, 1) && salloc(s, &s->Xb, bt * s->gm.k1) && salloc(s, &s->A1, bt * SUR_HID) &&
            salloc(s, &s->G2, bt * SUR_HID) && salloc(s, &s->G1, bt * SUR_HID) && salloc(s, &s->yb, bt) &&
            salloc(s, &s->Z1, bt * SUR_HID) && salloc(s, &s->Z2, bt * SUR_HID) && salloc(s, &s->loss_scratch, 1) &&
            salloc(s, &s->fit_acc, 2) && salloc(s, &s->err, 1) && salloc(s, &s->T, (size_t)cfg->max_pixels) &&
            (s->gm.dim == 2 || salloc(s, &s->wbuf, 4 * (size_t)cfg->max_pixels));
  if (!ok) {
    sfree(s);
    delete s;
    return PCSIR_ENOMEM;
  }
  const double norm0[2] = {0.0, 1.0};
  e = cudaMemset(s->P, 0, s->gm.ndev * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->G, 0, s->gm.ndev * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->Mo, 0, s->gm.ndev * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->V, 0, s->gm.ndev * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->W1b, 0, (size_t)SUR_HID * s->gm.k1 * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMemset(s->W2b, 0, (size_t)SUR_HID * SUR_HID * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMemset(s->Wsw, 0, (size_t)(s->gm.k1 / MM_K + SUR_HID / MM_K) * SI_W);
  if (e == cudaSuccess) e = cudaMemcpy(s->norm, norm0, sizeof(norm0), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->count, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(s->add_done, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(s->err, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    sfree(s);
    delete s;
    return PCSIR_ECUDA;
  }
  *out = s;
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_destroy(pcsir_surrogate* s) {
  if (!s) return PCSIR_OK;
  cudaDeviceSynchronize();
  sfree(s);
  delete s;
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_init(pcsir_surrogate* s, uint64_t seed, void* stream) {
  if (!s) return PCSIR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_sur_init<<<grid_for(s->gm.ndev, 256, s->num_sms), 256, 0, st>>>(s->P, (unsigned long long)seed, s->gm);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_sur_tobf16<<<grid_for((long long)SUR_HID * (s->gm.k1 + SUR_HID), 256, s->num_sms), 256, 0, st>>>(s->P, s->W1b,
                                                                                                     s->W2b, s->gm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = pack_weights(s, st);
  const double norm0[2] = {0.0, 1.0};
  if (e == cudaSuccess) e = cudaMemsetAsync(s->G, 0, s->gm.ndev * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->Mo, 0, s->gm.ndev * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->V, 0, s->gm.ndev * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemcpy(s->norm, norm0, sizeof(norm0), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return scuda(s, e, "surrogate initialisation");
  s->host_mean = 0.0;
  s->host_scale = 1.0;
  s->adam_t = 0;
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_set_params(pcsir_surrogate* s, const float* params, double label_mean,
                                        double label_scale) {
  if (!s || !params || !std::isfinite(label_mean) || !(label_scale > 0.0) || !std::isfinite(label_scale))
    return PCSIR_EINVAL;
  std::vector<float> dev((size_t)s->gm.ndev, 0.0f);
  const float* p = params;
  for (int r = 0; r < SUR_HID; ++r)
    for (int k = 0; k < s->gm.nin; ++k) dev[(size_t)(s->gm.off_w1 + r * s->gm.k1 + k)] = *p++;
  for (long long i = s->gm.off_b1; i < s->gm.ndev; ++i) dev[(size_t)i] = *p++;
  const double norm[2] = {label_mean, label_scale};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(s->P, dev.data(), s->gm.ndev * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->norm, norm, sizeof(norm), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->G, 0, s->gm.ndev * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->Mo, 0, s->gm.ndev * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->V, 0, s->gm.ndev * sizeof(float));
  if (e == cudaSuccess) {
    k_sur_tobf16<<<grid_for((long long)SUR_HID * (s->gm.k1 + SUR_HID), 256, s->num_sms), 256>>>(s->P, s->W1b, s->W2b, s->gm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = pack_weights(s, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return scuda(s, e, "setting surrogate parameters");
  s->host_mean = label_mean;
  s->host_scale = label_scale;
  s->adam_t = 0;
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_get_params(pcsir_surrogate* s, float* params, double* label_mean, double* label_scale) {
  if (!s || !params) return PCSIR_EINVAL;
  std::vector<float> dev((size_t)s->gm.ndev);
  double norm[2];
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(dev.data(), s->P, s->gm.ndev * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(norm, s->norm, sizeof(norm), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return scuda(s, e, "reading surrogate parameters");
  float* p = params;
  for (int r = 0; r < SUR_HID; ++r)
    for (int k = 0; k < s->gm.nin; ++k) *p++ = dev[(size_t)(s->gm.off_w1 + r * s->gm.k1 + k)];
  for (long long i = s->gm.off_b1; i < s->gm.ndev; ++i) *p++ = dev[(size_t)i];
  if (label_mean) *label_mean = norm[0];
  if (label_scale) *label_scale = norm[1];
  return PCSIR_OK;
}

}  // extern "C"

namespace {

pcsir_status sur_add(pcsir_surrogate* s, const double* dummy, int64_t stride, int64_t n, const double* ll,
                     double label_floor, const float* image, int32_t W, int32_t H, int32_t D, double bg,
                     double psf_sigma, void* stream) {
  if (!s) return PCSIR_EINVAL;
  if (n < 0 || W < 1 || H < 1 || D < 1 || stride < n || !std::isfinite(bg) || !(psf_sigma > 0.0) ||
      std::isnan(label_floor) || label_floor == INFINITY)
    return sfail(s, PCSIR_EINVAL, "invalid sizes or model parameters");
  if (n == 0) return PCSIR_OK;
  if (!dummy || !ll || !image) return sfail(s, PCSIR_EINVAL, "NULL device pointer");
  const long long blocks = (n + ADD_THREADS - 1) / ADD_THREADS;
  if (blocks > s->add_max_blocks) return sfail(s, PCSIR_ERANGE, "more than 2^20 states in one call");
  if ((long long)W * H * D > s->cfg.max_pixels) return sfail(s, PCSIR_ERANGE, "image larger than max_pixels");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_window(s, image, W, H, D, bg, st);
  if (e == cudaSuccess) {
    k_sur_add_count<<<(unsigned)blocks, ADD_THREADS, 0, st>>>(s->gm, dummy, stride, n, W, H, D, s->add_cnt,
                                                              s->count, s->add_base);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_sur_add_write<<<(unsigned)blocks, ADD_THREADS, 0, st>>>(s->gm, dummy, stride, n, ll, label_floor, s->T, image,
                                                              W, H, D, make_feat(s, bg, psf_sigma), s->add_cnt,
                                                              s->add_base, s->count, s->add_done, s->cfg.capacity,
                                                              s->X, s->y, s->cens);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return scuda(s, e, "dataset append");
  return PCSIR_OK;
}

pcsir_status sur_predict(pcsir_surrogate* s, const double* dummy, int64_t stride, int64_t n, const float* image,
                         int32_t W, int32_t H, int32_t D, double bg, double psf_sigma, double* out, void* stream) {
  if (!s) return PCSIR_EINVAL;
  if (n < 0 || W < 1 || H < 1 || D < 1 || stride < n || !std::isfinite(bg) || !(psf_sigma > 0.0))
    return sfail(s, PCSIR_EINVAL, "invalid sizes or model parameters");
  if (n == 0) return PCSIR_OK;
  if (!dummy || !image || !out) return sfail(s, PCSIR_EINVAL, "NULL device pointer");
  if ((long long)W * H * D > s->cfg.max_pixels) return sfail(s, PCSIR_ERANGE, "image larger than max_pixels");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t ew = launch_window(s, image, W, H, D, bg, st);
  if (ew != cudaSuccess) return scuda(s, ew, "window terms");
  SurInfer a{};
  a.net = net_of(s);
  a.gm = s->gm;
  a.dummy = dummy;
  a.stride = stride;
  a.n = n;
  a.img = image;
  a.W = W;
  a.H = H;
  a.D = D;
  a.sf = make_feat(s, bg, psf_sigma);
  a.T = s->T;
  a.out = out;
  a.nan_clipped = 1;
  a.err = s->err;
  const cudaError_t e = launch_infer(s, a, SRC_STATES, (n + 127) / 128, st);
  if (e != cudaSuccess) return scuda(s, e, "surrogate inference");
  return PCSIR_OK;
}

}  // namespace

extern "C" {

pcsir_status pcsir_surrogate_add(pcsir_surrogate* s, const double* dummy, int64_t stride, int64_t n, const double* ll,
                                 double label_floor, const float* image, int32_t W, int32_t H, double bg,
                                 double psf_sigma, void* stream) {
  if (s && s->gm.dim != 2) return sfail(s, PCSIR_EINVAL, "a 3D surrogate takes pcsir_surrogate_add3");
  return sur_add(s, dummy, stride, n, ll, label_floor, image, W, H, 1, bg, psf_sigma, stream);
}

pcsir_status pcsir_surrogate_add3(pcsir_surrogate* s, const double* dummy, int64_t stride, int64_t n,
                                  const double* ll, double label_floor, const float* volume, int32_t W, int32_t H,
                                  int32_t D, double bg, double psf_sigma_xy, void* stream) {
  if (s && s->gm.dim != 3) return sfail(s, PCSIR_EINVAL, "a 2D surrogate takes pcsir_surrogate_add");
  return sur_add(s, dummy, stride, n, ll, label_floor, volume, W, H, D, bg, psf_sigma_xy, stream);
}

pcsir_status pcsir_surrogate_rows(pcsir_surrogate* s, int64_t* rows) {
  if (!s || !rows) return PCSIR_EINVAL;
  unsigned long long c = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&c, s->count, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return scuda(s, e, "reading the row count");
  *rows = (int64_t)c;
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_clear(pcsir_surrogate* s, void* stream) {
  if (!s) return PCSIR_EINVAL;
  cudaError_t e = cudaMemsetAsync(s->count, 0, sizeof(unsigned long long), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return scuda(s, e, "clearing the dataset");
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_dataset(pcsir_surrogate* s, const uint16_t** inputs, const float** labels,
                                     const uint8_t** censored) {
  if (!s || !inputs || !labels || !censored) return PCSIR_EINVAL;
  *inputs = reinterpret_cast<const uint16_t*>(s->X);
  *labels = s->y;
  *censored = s->cens;
  return PCSIR_OK;
}

static pcsir_status check_range(pcsir_surrogate* s, int64_t begin, int64_t end) {
  int64_t rows = 0;
  pcsir_status st = pcsir_surrogate_rows(s, &rows);
  if (st != PCSIR_OK) return st;
  if (begin < 0 || end <= begin || end > rows) return sfail(s, PCSIR_EINVAL, "row range outside the dataset");
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_fit_scale(pcsir_surrogate* s, int64_t begin, int64_t end) {
  if (!s) return PCSIR_EINVAL;
  pcsir_status ps = check_range(s, begin, end);
  if (ps != PCSIR_OK) return ps;
  const long long n = end - begin;
  double acc[2];
  // first pass: mean; second: variance about the mean
  cudaError_t e = cudaMemset(s->fit_acc, 0, 2 * sizeof(double));
  if (e == cudaSuccess) {
    k_sur_sums<<<grid_for(n, 256, s->num_sms), 256>>>(s->y, begin, end, 0.0, s->fit_acc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(acc, s->fit_acc, sizeof(acc), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return scuda(s, e, "label sums");
  const double mean = acc[0] / (double)n;
  e = cudaMemset(s->fit_acc, 0, 2 * sizeof(double));
  if (e == cudaSuccess) {
    k_sur_sums<<<grid_for(n, 256, s->num_sms), 256>>>(s->y, begin, end, mean, s->fit_acc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(acc, s->fit_acc, sizeof(acc), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return scuda(s, e, "label sums");
  double scale = std::sqrt(acc[1] / (double)n);
  if (!(scale > 0.0) || !std::isfinite(scale)) scale = 1.0;
  const double norm[2] = {mean, scale};
  e = cudaMemcpy(s->norm, norm, sizeof(norm), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return scuda(s, e, "label normalisation");
  s->host_mean = mean;
  s->host_scale = scale;
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_train(pcsir_surrogate* s, int64_t begin, int64_t end, int32_t steps, double lr,
                                   uint64_t seed, float* loss, void* stream) {
  if (!s) return PCSIR_EINVAL;
  if (steps < 0 || !(lr > 0.0) || !std::isfinite(lr)) return sfail(s, PCSIR_EINVAL, "invalid steps or rate");
  pcsir_status ps = check_range(s, begin, end);
  if (ps != PCSIR_OK) return ps;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int bt = s->cfg.batch;
  const long long range = end - begin;
  cudaError_t e = cudaSuccess;
  if (loss) e = cudaMemsetAsync(loss, 0, (size_t)steps * sizeof(float), st);
  for (int k = 0; k < steps && e == cudaSuccess; ++k) {
    const long long step = s->adam_t;
    k_sur_gather<<<(bt + 7) / 8, 256, 0, st>>>(s->X, s->y, s->cens, begin, range, (unsigned long long)seed, step,
                                              bt, s->norm, s->Xb, s->yb, s->cb, s->gm.k1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = fwd_bwd(s, bt, loss ? loss + k : nullptr, st);
    if (e != cudaSuccess) break;
    s->adam_t += 1;
    const double t = (double)s->adam_t;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, t)));
    k_sur_adam<<<grid_for(s->gm.ndev, 256, s->num_sms), 256, 0, st>>>(s->P, s->G, s->Mo, s->V, (float)lr, c1, c2, s->W1b,
                                                               s->W2b, s->gm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && steps > 0) e = pack_weights(s, st);
  if (e != cudaSuccess) return scuda(s, e, "training step");
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_grads(pcsir_surrogate* s, int64_t begin, int32_t n, float* grads, double* loss) {
  if (!s || !grads) return PCSIR_EINVAL;
  if (n < 128 || n > s->cfg.batch || (n % 128) != 0) return sfail(s, PCSIR_EINVAL, "n must be a multiple of 128 <= batch");
  pcsir_status ps = check_range(s, begin, begin + n);
  if (ps != PCSIR_OK) return ps;
  cudaError_t e = cudaMemset(s->G, 0, s->gm.ndev * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->loss_scratch, 0, sizeof(float));
  if (e == cudaSuccess) {
    // rows in order: update index 0 takes rows begin .. begin + n - 1
    k_sur_gather<<<(n + 7) / 8, 256>>>(s->X, s->y, s->cens, begin, n, 0ull, 0, n, s->norm, s->Xb, s->yb, s->cb, s->gm.k1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = fwd_bwd(s, n, s->loss_scratch, 0);
  std::vector<float> dev((size_t)s->gm.ndev);
  float l = 0.0f;
  if (e == cudaSuccess) e = cudaMemcpy(dev.data(), s->G, s->gm.ndev * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&l, s->loss_scratch, sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(s->G, 0, s->gm.ndev * sizeof(float));
  if (e != cudaSuccess) return scuda(s, e, "gradient pass");
  float* p = grads;
  for (int r = 0; r < SUR_HID; ++r)
    for (int k = 0; k < s->gm.nin; ++k) *p++ = dev[(size_t)(s->gm.off_w1 + r * s->gm.k1 + k)];
  for (long long i = s->gm.off_b1; i < s->gm.ndev; ++i) *p++ = dev[(size_t)i];
  if (loss) *loss = (double)l;
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_predict_rows(pcsir_surrogate* s, int64_t begin, int64_t end, double* out,
                                          void* stream) {
  if (!s || !out) return PCSIR_EINVAL;
  pcsir_status ps = check_range(s, begin, end);
  if (ps != PCSIR_OK) return ps;
  SurInfer a{};
  a.net = net_of(s);
  a.gm = s->gm;
  a.D = 1;
  a.rows = s->X + (size_t)begin * s->gm.k1;
  a.n = end - begin;
  a.out = out;
  a.err = s->err;
  const cudaError_t e = launch_infer(s, a, SRC_ROWS, (a.n + 127) / 128, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return scuda(s, e, "surrogate inference");
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_predict(pcsir_surrogate* s, const double* dummy, int64_t stride, int64_t n,
                                     const float* image, int32_t W, int32_t H, double bg, double psf_sigma,
                                     double* out, void* stream) {
  if (s && s->gm.dim != 2) return sfail(s, PCSIR_EINVAL, "a 3D surrogate takes pcsir_surrogate_predict3");
  return sur_predict(s, dummy, stride, n, image, W, H, 1, bg, psf_sigma, out, stream);
}

pcsir_status pcsir_surrogate_predict3(pcsir_surrogate* s, const double* dummy, int64_t stride, int64_t n,
                                      const float* volume, int32_t W, int32_t H, int32_t D, double bg,
                                      double psf_sigma_xy, double* out, void* stream) {
  if (s && s->gm.dim != 3) return sfail(s, PCSIR_EINVAL, "a 2D surrogate takes pcsir_surrogate_predict");
  return sur_predict(s, dummy, stride, n, volume, W, H, D, bg, psf_sigma_xy, out, stream);
}

pcsir_status pcsir_surrogate_nparams(pcsir_surrogate* s, int64_t* nparams) {
  if (!s || !nparams) return PCSIR_EINVAL;
  *nparams = (int64_t)SUR_HID * s->gm.nin + (s->gm.ndev - s->gm.off_b1);
  return PCSIR_OK;
}

}  // extern "C"
