// Fifth-generation tensor core (tcgen05) building blocks for sm_103a: shared
// memory matrix descriptors, the instruction descriptor of kind::f16 with
// FP32 accumulation, TMEM allocation, MMA issue and commit to an mbarrier,
// bounded mbarrier waits, TMEM loads, and the staging of bf16 operands into
// the 128-byte-swizzled K-major layout.
//
// Operand layout in shared memory (K-major, 128-byte swizzle): a 64-wide K
// chunk of R rows is R rows of 128 bytes; within each group of 8 rows (1024
// bytes, SBO) the 16-byte pieces of row r are permuted by XOR with r mod 8,
// so that the eight rows of a core matrix fall in different banks.  A chunk
// starts on a 1024-byte boundary.  One tcgen05.mma consumes K = 16, and the
// descriptor of the s-th K = 16 step of a chunk starts 32 * s bytes after it
// (the swizzle is applied to the computed addresses).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

#include "pcsir_internal.h"

namespace pcsir {

constexpr int MM_K = 64;  // K per staged chunk
constexpr uint32_t MM_SBO = 1024;
constexpr int MM_WAIT_SPINS = 1 << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4, leading offset 1 (unused for
// swizzled K-major operands), SBO >> 4, version 1, base offset 0, 128-byte
// swizzle (mode 2)
__device__ __forceinline__ uint64_t mm_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(MM_SBO >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t mm_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) of a staged K chunk
__device__ __forceinline__ uint32_t mm_off(int r, int k) {
  return (uint32_t)(r * 128 + ((((k >> 3) ^ r) & 7) << 4) + (k & 7) * 2);
}

// first 1024-byte boundary at or after p (shared memory)
__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  const uint32_t a = smem_u32(p);
  return p + (((a + 1023u) & ~1023u) - a);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait for the mbarrier phase; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  const uint32_t a = smem_u32(bar);
  for (int i = 0; i < MM_WAIT_SPINS; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Issue the four K = 16 MMAs of one staged 64-wide K chunk (one thread).
__device__ __forceinline__ void tc_mma_chunk(uint32_t tmem, uint32_t a0, uint32_t b0, uint32_t idesc, bool first) {
#pragma unroll
  for (int s = 0; s < MM_K / 16; ++s)
    tc_mma(tmem, mm_desc(a0 + s * 32), mm_desc(b0 + s * 32), idesc, (!first || s > 0) ? 1u : 0u);
}

__device__ __forceinline__ uint4 pack_bf16x8(const float v[8]) {
  uint4 u;
  u.x = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[0])) |
        ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[1])) << 16);
  u.y = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2])) |
        ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[3])) << 16);
  u.z = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[4])) |
        ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[5])) << 16);
  u.w = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[6])) |
        ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[7])) << 16);
  return u;
}

__device__ __forceinline__ float silu_f(float t) { return t / (1.0f + __expf(-t)); }
__device__ __forceinline__ float silu_grad_f(float t) {
  const float s = 1.0f / (1.0f + __expf(-t));
  return s * (1.0f + t * (1.0f - s));
}

// Stage a rows x 64 chunk of an operand, element (r, k) = src[(r0 + r) srow +
// (k0 + k) sk], into the swizzled layout; rows >= rows_valid and k >= K are
// zero.  Three access patterns: K contiguous (sk == 1, 16-byte loads), rows
// contiguous (srow == 1, lanes over rows), and any other strides.  Each
// thread issues all its loads before its shared-memory stores, so their
// latencies overlap.
__device__ __forceinline__ uint4 mm_load8(const __nv_bfloat16* src, long long srow, long long sk, int row,
                                          int rows_valid, int kk, int K) {
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (row < rows_valid) {
    const __nv_bfloat16* p = src + (long long)row * srow + (long long)kk * sk;
    if (sk == 1 && kk + 8 <= K && ((reinterpret_cast<uintptr_t>(p) & 15u) == 0u)) {
      v = __ldg(reinterpret_cast<const uint4*>(p));
    } else {
      unsigned short e[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        e[i] = (kk + i < K) ? __bfloat16_as_ushort(p[(long long)i * sk]) : (unsigned short)0;
      v.x = e[0] | ((unsigned)e[1] << 16);
      v.y = e[2] | ((unsigned)e[3] << 16);
      v.z = e[4] | ((unsigned)e[5] << 16);
      v.w = e[6] | ((unsigned)e[7] << 16);
    }
  }
  return v;
}

// A thread's share of one staged chunk: its 8-element groups, loaded into registers (mm_fetch) and
// written to the swizzled layout later (mm_put), so that the loads of the next chunk can be in
// flight while the tensor core works on the current one.
template <int NTHREADS, int NROWS>
struct MmFrag {
  static constexpr int PER = NROWS * (MM_K / 8) / NTHREADS;  // 8-element groups per thread
  static_assert(PER * NTHREADS == NROWS * (MM_K / 8), "tile not divisible among threads");
  uint4 v[PER];
};

__device__ __forceinline__ void mm_group(int g, int nrows, bool mn_major, int* r, int* kg) {
  if (mn_major) {
    *r = g % nrows;
    *kg = (g / nrows) * 8;
  } else {
    *r = g / (MM_K / 8);
    *kg = (g % (MM_K / 8)) * 8;
  }
}

template <int NTHREADS, int NROWS>
__device__ __forceinline__ void mm_fetch(MmFrag<NTHREADS, NROWS>& f, const __nv_bfloat16* src, long long srow,
                                         long long sk, int r0, int rows_valid, int k0, int K) {
  const bool mn_major = (srow == 1 && sk != 1);
#pragma unroll
  for (int j = 0; j < MmFrag<NTHREADS, NROWS>::PER; ++j) {
    int r, kg;
    mm_group(threadIdx.x + j * NTHREADS, NROWS, mn_major, &r, &kg);
    f.v[j] = mm_load8(src, srow, sk, r0 + r, rows_valid, k0 + kg, K);
  }
}

template <int NTHREADS, int NROWS>
__device__ __forceinline__ void mm_put(uint8_t* dst, const MmFrag<NTHREADS, NROWS>& f, long long srow, long long sk) {
  const bool mn_major = (srow == 1 && sk != 1);
#pragma unroll
  for (int j = 0; j < MmFrag<NTHREADS, NROWS>::PER; ++j) {
    int r, kg;
    mm_group(threadIdx.x + j * NTHREADS, NROWS, mn_major, &r, &kg);
    *reinterpret_cast<uint4*>(dst + mm_off(r, kg)) = f.v[j];
  }
}

template <int NTHREADS, int NROWS>
__device__ __forceinline__ void mm_stage(uint8_t* dst, const __nv_bfloat16* src, long long srow, long long sk,
                                         int r0, int rows_valid, int k0, int K) {
  MmFrag<NTHREADS, NROWS> f;
  mm_fetch(f, src, srow, sk, r0, rows_valid, k0, K);
  mm_put(dst, f, srow, sk);
}

// ---------------------------------------------------------------------------
// Generic GEMM (pcsir_mlp.cu):
//   acc[m, n] = sum_k A(m, k) B(n, k),  A(m, k) = A[m sam + k sak], B(n, k) = B[n sbn + k sbk]
// with one of the epilogues below.  Split K (kchunks_per_split > 0) runs
// gridDim.z slices of the K chunks and needs EPI_ATOMIC.
// ---------------------------------------------------------------------------
enum {
  EPI_STORE = 0,   // C[m, n] = acc (+ C[m, n] if accumulate)
  EPI_ATOMIC = 1,  // C[m, n] += acc with atomics (split K)
  EPI_ACT = 2,     // pre = acc + bias[n]; C[m, n] = pre (if C); act[m, n] = bf16(silu(pre))
  EPI_DACT = 3,    // v = acc * silu'(pre[m, n]); act[m, n] = bf16(v); colsum[n] += sum over m of v
};

struct GemmArgs {
  const __nv_bfloat16* A;
  long long sam, sak;
  const __nv_bfloat16* B;
  long long sbn, sbk;
  float* C;
  long long ldc;
  int M, N, K;
  int accumulate;
  int epi;
  int kchunks_per_split;  // 0: no split
  const float* bias;
  __nv_bfloat16* act;
  long long ld_act;
  const float* pre;
  long long ld_pre;
  float* colsum;
  unsigned* err;
};

cudaError_t prepare_gemm();
// nt: column tile (64 or 256; 0 picks one); splits: K slices (1 = none)
cudaError_t launch_gemm(GemmArgs g, cudaStream_t s, int nt = 0, int splits = 1);

}  // namespace pcsir
