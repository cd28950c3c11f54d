// BF16 tensor-core GEMM on sm_103a with the fifth-generation tensor core
// instructions (tcgen05): operands staged in shared memory, one thread issues
// tcgen05.mma with FP32 accumulation in tensor memory (TMEM), completion
// through tcgen05.commit to an mbarrier, results read back with tcgen05.ld.
// This is the building block of the likelihood surrogate's training and
// inference.
//
//   C[m, n] (+)= sum_k A(m, k) B(n, k),   A(m, k) = A[m sam + k sak],
//                                         B(n, k) = B[n sbn + k sbk]   (bf16)
// with an optional epilogue (bias, SiLU, bf16 copies of the activation and of
// its transpose) used by the network's layers.
//
// Shared-memory operand layout (no swizzle, K-major): 8 x 8 bf16 "core
// matrices" of 128 contiguous bytes (8 rows of 16 bytes); cores adjacent along
// K are LBO = 128 bytes apart, 8-row groups are SBO = 1024 bytes apart, so a
// 64-wide K chunk of 128 rows is 16 KB.  One tcgen05.mma consumes K = 16 (two
// cores along K).
#include <cstdint>
#include <cuda_bf16.h>

#include "pcsir_device.cuh"

namespace pcsir {

constexpr int MM_M = 128;        // rows per CTA tile (TMEM lanes)
constexpr int MM_K = 64;         // K per staged chunk
constexpr int MM_THREADS = 128;  // four warps: one TMEM lane quarter each
constexpr uint32_t MM_LBO = 128;
constexpr uint32_t MM_SBO = 1024;
constexpr int MM_WAIT_SPINS = 1 << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, LBO, SBO (all >> 4), version 1,
// no swizzle
__device__ __forceinline__ uint64_t mm_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(MM_LBO >> 4) << 16) | ((uint64_t)(MM_SBO >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t mm_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) of a staged K-chunk
__device__ __forceinline__ uint32_t mm_off(int r, int k) {
  return (uint32_t)((r >> 3) * MM_SBO + (k >> 3) * MM_LBO + (r & 7) * 16 + (k & 7) * 2);
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

// Epilogue of a GEMM tile (row m, columns n0 + j):
//   EPI_STORE : C[m, n] = acc (+ C[m, n] if accumulate)
//   EPI_ACT   : pre = acc + bias[n]; C[m, n] = pre (fp32); act[m, n] = bf16(silu(pre));
//               actT[n, m] = same (transposed copy, leading dimension ldt)
enum { EPI_STORE = 0, EPI_ACT = 1 };

struct GemmArgs {
  const __nv_bfloat16* A;
  long long sam, sak;
  const __nv_bfloat16* B;
  long long sbn, sbk;
  float* C;
  long long ldc;
  int M, N, K;
  int accumulate;  // add to the existing C (EPI_STORE)
  int epi;
  const float* bias;
  __nv_bfloat16* act;
  long long lda_act;
  __nv_bfloat16* actT;
  long long ldt;
  unsigned* err;
};

__device__ __forceinline__ float silu(float x) { return x / (1.0f + __expf(-x)); }

// Stage a rows x 64 chunk of an operand (rows r0.., K k0..) into the core-matrix layout;
// out-of-range elements are zero.
__device__ __forceinline__ void mm_stage(uint8_t* dst, const __nv_bfloat16* src, long long srow, long long sk,
                                         int r0, int nrows_tile, int rows_valid, int k0, int K) {
  const int tid = threadIdx.x;
  const int total = nrows_tile * (MM_K / 8);  // 8-element groups along K
  for (int g = tid; g < total; g += MM_THREADS) {
    const int r = g / (MM_K / 8);
    const int kg = (g % (MM_K / 8)) * 8;
    const int row = r0 + r;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (row < rows_valid) {
      const int kk = k0 + kg;
      const __nv_bfloat16* p = src + (long long)row * srow + (long long)kk * sk;
      if (sk == 1 && kk + 8 <= K && ((reinterpret_cast<uintptr_t>(p) & 15u) == 0u)) {
        v = *reinterpret_cast<const uint4*>(p);
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
    *reinterpret_cast<uint4*>(dst + mm_off(r, kg)) = v;
  }
}

// One CTA: rows [m0, m0 + 128) x columns [n0, n0 + NT).
template <int NT>
__global__ void __launch_bounds__(MM_THREADS) k_gemm_bf16(GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t mm_smem[];
  uint8_t* sA = mm_smem;                              // 128 x 64 bf16 = 16 KB
  uint8_t* sB = mm_smem + MM_M * MM_K * 2;            // NT x 64 bf16
  uint64_t* bar = reinterpret_cast<uint64_t*>(mm_smem + MM_M * MM_K * 2 + NT * MM_K * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * MM_M;
  const int n0 = blockIdx.y * NT;
  constexpr uint32_t NCOLS = NT < 32 ? 32 : NT;
  if (warp == 0) tc_alloc(tslot, NCOLS);
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = mm_idesc(MM_M, NT);
  uint32_t phase = 0;
  bool ok = true;
  const int nk = (g.K + MM_K - 1) / MM_K;
  for (int kc = 0; kc < nk && ok; ++kc) {
    mm_stage(sA, g.A, g.sam, g.sak, m0, MM_M, g.M, kc * MM_K, g.K);
    mm_stage(sB, g.B, g.sbn, g.sbk, n0, NT, g.N, kc * MM_K, g.K);
    proxy_fence();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int s = 0; s < MM_K / 16; ++s)
        tc_mma(tmem, mm_desc(a0 + s * 2 * MM_LBO), mm_desc(b0 + s * 2 * MM_LBO), idesc, (kc > 0 || s > 0) ? 1u : 0u);
      tc_commit(bar);
    }
    // every thread waits; the block continues only if all saw the phase complete
    ok = __syncthreads_and(mbar_wait(bar, phase) ? 1 : 0) != 0;
    phase ^= 1u;
    tc_fence_after();
  }
  if (!ok) {
    if (tid == 0) atomicOr(g.err, (unsigned)PCSIR_DERR_TIMEOUT);
  } else {
    // epilogue: thread tid owns TMEM lane (row) tid
    const int m = m0 + tid;
    for (int c = 0; c < NT; c += 8) {
      float v[8];
      tc_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      if (m < g.M) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int n = n0 + c + i;
          if (n >= g.N) continue;
          float* cp = g.C + (long long)m * g.ldc + n;
          if (g.epi == EPI_STORE) {
            *cp = g.accumulate ? *cp + v[i] : v[i];
          } else {
            const float pre = v[i] + g.bias[n];
            *cp = pre;
            const __nv_bfloat16 a = __float2bfloat16_rn(silu(pre));
            if (g.act) g.act[(long long)m * g.lda_act + n] = a;
            if (g.actT) g.actT[(long long)n * g.ldt + m] = a;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, NCOLS);
}

template <int NT>
static size_t gemm_smem() {
  return (size_t)MM_M * MM_K * 2 + (size_t)NT * MM_K * 2 + 16 + 1024;
}

cudaError_t prepare_gemm() {
  // leave room for at most two CTAs per SM, so two tiles of 256 TMEM columns fit
  const int want = 100 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_bf16<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
  return e;
}

cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t s) {
  const size_t smem = 100 * 1024;  // >= gemm_smem<256>() (49 KB): caps residency at two CTAs per SM
  if (g.N > 64) {
    dim3 grid((g.M + MM_M - 1) / MM_M, (g.N + 255) / 256);
    k_gemm_bf16<256><<<grid, MM_THREADS, smem, s>>>(g);
  } else {
    dim3 grid((g.M + MM_M - 1) / MM_M, (g.N + 63) / 64);
    k_gemm_bf16<64><<<grid, MM_THREADS, smem, s>>>(g);
  }
  return cudaGetLastError();
}

}  // namespace pcsir

using namespace pcsir;

namespace {
unsigned* g_gemm_err = nullptr;
}

extern "C" pcsir_status pcsir_gemm_bf16(const uint16_t* A, int64_t sam, int64_t sak, const uint16_t* B, int64_t sbn,
                                        int64_t sbk, float* C, int64_t ldc, int32_t M, int32_t N, int32_t K,
                                        int32_t accumulate, void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1) return PCSIR_EINVAL;
  static bool prepared = false;
  if (!prepared) {
    if (prepare_gemm() != cudaSuccess) return PCSIR_ECUDA;
    if (cudaMalloc(&g_gemm_err, sizeof(unsigned)) != cudaSuccess) return PCSIR_ENOMEM;
    cudaMemset(g_gemm_err, 0, sizeof(unsigned));
    prepared = true;
  }
  GemmArgs g{};
  g.A = reinterpret_cast<const __nv_bfloat16*>(A);
  g.sam = sam;
  g.sak = sak;
  g.B = reinterpret_cast<const __nv_bfloat16*>(B);
  g.sbn = sbn;
  g.sbk = sbk;
  g.C = C;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.accumulate = accumulate;
  g.epi = EPI_STORE;
  g.err = g_gemm_err;
  return launch_gemm(g, static_cast<cudaStream_t>(stream)) == cudaSuccess ? PCSIR_OK : PCSIR_ECUDA;
}
