// BF16 tensor-core GEMM on sm_103a (tcgen05): operands staged in shared
// memory, one thread issues tcgen05.mma with FP32 accumulation in tensor
// memory (TMEM), completion through tcgen05.commit to an mbarrier, results
// read back with tcgen05.ld.  The training passes of the likelihood surrogate
// are built from it (forward layers with a bias + SiLU epilogue, the
// backward product through the SiLU derivative, and split-K weight
// gradients).
#include <algorithm>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>

#include "pcsir_device.cuh"
#include "pcsir_tc.cuh"

namespace pcsir {

constexpr int MM_M = 128;        // rows per CTA tile (TMEM lanes)
constexpr int MM_THREADS = 128;  // four warps: one TMEM lane quarter each

// Epilogue of a finished tile: thread tid owns TMEM lane (row) tid.
template <int NT>
__device__ __forceinline__ void gemm_epilogue(const GemmArgs& g, uint32_t tmem, int m0, int n0) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = m0 + tid;
  const bool mrow = m < g.M;
  for (int c = 0; c < NT; c += 8) {
    float v[8];
    tc_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
    if (g.epi == EPI_DACT) {
      float cs[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int n = n0 + c + i;
        float d = 0.0f;
        if (mrow && n < g.N) d = v[i] * silu_grad_f(g.pre[(long long)m * g.ld_pre + n]);
        v[i] = d;
        cs[i] = d;
      }
      if (mrow) {
        if (n0 + c + 8 <= g.N && (g.ld_act % 8) == 0) {
          *reinterpret_cast<uint4*>(g.act + (long long)m * g.ld_act + n0 + c) = pack_bf16x8(v);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (n0 + c + i < g.N) g.act[(long long)m * g.ld_act + n0 + c + i] = __float2bfloat16_rn(v[i]);
        }
      }
      if (g.colsum) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float s = cs[i];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0 && n0 + c + i < g.N) atomicAdd(g.colsum + n0 + c + i, s);
        }
      }
      continue;
    }
    if (!mrow) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int n = n0 + c + i;
      if (n >= g.N) continue;
      float* cp = g.C ? g.C + (long long)m * g.ldc + n : nullptr;
      if (g.epi == EPI_STORE) {
        *cp = g.accumulate ? *cp + v[i] : v[i];
      } else if (g.epi == EPI_ATOMIC) {
        atomicAdd(cp, v[i]);
      } else {  // EPI_ACT
        const float pre = v[i] + g.bias[n];
        if (cp) *cp = pre;
        v[i] = silu_f(pre);
      }
    }
    if (g.epi == EPI_ACT && g.act) {
      if (n0 + c + 8 <= g.N && (g.ld_act % 8) == 0) {
        *reinterpret_cast<uint4*>(g.act + (long long)m * g.ld_act + n0 + c) = pack_bf16x8(v);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (n0 + c + i < g.N) g.act[(long long)m * g.ld_act + n0 + c + i] = __float2bfloat16_rn(v[i]);
      }
    }
  }
}

// One CTA: rows [m0, m0 + 128) x columns [n0, n0 + NT), K chunks of its slice.
template <int NT>
__global__ void __launch_bounds__(MM_THREADS) k_gemm_bf16(GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t mm_smem_raw[];
  uint8_t* mm_smem = align1024(mm_smem_raw);
  uint8_t* sA = mm_smem;                    // 128 x 64 bf16 = 16 KB
  uint8_t* sB = mm_smem + MM_M * MM_K * 2;  // NT x 64 bf16
  uint64_t* bar = reinterpret_cast<uint64_t*>(mm_smem + MM_M * MM_K * 2 + NT * MM_K * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * MM_M;
  const int n0 = blockIdx.y * NT;
  const int nk_total = (g.K + MM_K - 1) / MM_K;
  int kc0 = 0, kc1 = nk_total;
  if (g.kchunks_per_split > 0) {
    kc0 = blockIdx.z * g.kchunks_per_split;
    kc1 = min(nk_total, kc0 + g.kchunks_per_split);
  }
  if (kc0 >= kc1) return;  // empty K slice (uniform over the block)
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
  for (int kc = kc0; kc < kc1 && ok; ++kc) {
    mm_stage<MM_THREADS, MM_M>(sA, g.A, g.sam, g.sak, m0, g.M, kc * MM_K, g.K);
    mm_stage<MM_THREADS, NT>(sB, g.B, g.sbn, g.sbk, n0, g.N, kc * MM_K, g.K);
    proxy_fence();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      tc_mma_chunk(tmem, smem_u32(sA), smem_u32(sB), idesc, kc == kc0);
      tc_commit(bar);
    }
    // thread 0 polls the mbarrier (polling by every warp would compete with the
    // tensor core for shared memory); the block barrier releases the others
    ok = __syncthreads_and(tid != 0 || mbar_wait(bar, phase)) != 0;
    phase ^= 1u;
    tc_fence_after();
  }
  if (!ok) {
    if (tid == 0) atomicOr(g.err, (unsigned)PCSIR_DERR_TIMEOUT);
  } else {
    gemm_epilogue<NT>(g, tmem, m0, n0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, NCOLS);
}

// ---------------------------------------------------------------------------
// Multi-stage variant for operands whose K elements are contiguous (sak = sbk = 1, rows on 16-byte
// boundaries): each thread's 16-byte pieces of a K chunk go straight from global to their swizzled
// place in shared memory by cp.async (zero-filled past K and past the last row), S chunks in flight,
// so the tensor core does not wait for one chunk's loads after another.  Chunk kc + S - 1 is issued
// into the buffer chunk kc - 1 used once that chunk's MMAs have completed (its mbarrier).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// copies of a NROWS x 64 chunk (rows r0.., K from k0) of a K-contiguous operand into dst
template <int NROWS>
__device__ __forceinline__ void mm_async_chunk(uint32_t dst, const __nv_bfloat16* src, long long srow, int r0,
                                               int rows_valid, int k0, int K) {
  constexpr int PER = NROWS * (MM_K / 8) / MM_THREADS;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int gi = threadIdx.x + j * MM_THREADS;
    const int r = gi / (MM_K / 8), kg = (gi % (MM_K / 8)) * 8;
    const int row = r0 + r, k = k0 + kg;
    const int left = K - k;
    const uint32_t bytes = (row < rows_valid && left > 0) ? (uint32_t)(left >= 8 ? 16 : 2 * left) : 0u;
    // no byte is read when bytes == 0; the address stays a valid one all the same
    const __nv_bfloat16* p = bytes ? src + (long long)row * srow + k : src;
    cp_async16(dst + mm_off(r, kg), p, bytes);
  }
}

template <int NT, int S>
__global__ void __launch_bounds__(MM_THREADS) k_gemm_bf16_async(GemmArgs g) {
  static_assert(S >= 2 && S <= 4, "2 to 4 stages");
  extern __shared__ __align__(1024) uint8_t mm_smem_raw[];
  uint8_t* mm_smem = align1024(mm_smem_raw);
  constexpr int SA = MM_M * MM_K * 2, ST = SA + NT * MM_K * 2;  // one stage: A 16 KB, then B
  uint64_t* bar = reinterpret_cast<uint64_t*>(mm_smem + S * ST);  // one per stage
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + S);
  const uint32_t s0 = smem_u32(mm_smem);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * MM_M;
  const int n0 = blockIdx.y * NT;
  const int nk_total = (g.K + MM_K - 1) / MM_K;
  int kc0 = 0, kc1 = nk_total;
  if (g.kchunks_per_split > 0) {
    kc0 = blockIdx.z * g.kchunks_per_split;
    kc1 = min(nk_total, kc0 + g.kchunks_per_split);
  }
  if (kc0 >= kc1) return;  // empty K slice (uniform over the block)
  constexpr uint32_t NCOLS = NT < 32 ? 32 : NT;
  if (warp == 0) tc_alloc(tslot, NCOLS);
  if (tid == 0) {
#pragma unroll
    for (int j = 0; j < S; ++j) mbar_init(&bar[j], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = mm_idesc(MM_M, NT);
  auto issue = [&](int kc, int st) {
    mm_async_chunk<MM_M>(s0 + st * ST, g.A, g.sam, m0, g.M, kc * MM_K, g.K);
    mm_async_chunk<NT>(s0 + st * ST + SA, g.B, g.sbn, n0, g.N, kc * MM_K, g.K);
  };
#pragma unroll
  for (int j = 0; j < S - 1; ++j) {
    if (kc0 + j < kc1) issue(kc0 + j, j);
    cp_async_commit();
  }
  uint32_t phase[S];
#pragma unroll
  for (int j = 0; j < S; ++j) phase[j] = 0u;
  bool ok = true;
  for (int kc = kc0; kc < kc1 && ok; ++kc) {
    const int st = (kc - kc0) % S;
    cp_async_wait<S - 2>();  // this thread's pieces of chunk kc have landed
    proxy_fence();           // visible to the tensor core's reads
    __syncthreads();         // and everyone else's
    if (tid == 0) {
      tc_fence_after();
      tc_mma_chunk(tmem, s0 + st * ST, s0 + st * ST + SA, idesc, kc == kc0);
      tc_commit(&bar[st]);
    }
    const int kn = kc + S - 1;
    if (kn < kc1) {
      const int sn = (kn - kc0) % S;  // the stage chunk kc - 1 used
      if (kc > kc0) {
        // thread 0 polls the mbarrier (polling by every warp would compete with the tensor core
        // for shared memory); the block barrier releases the others
        ok = __syncthreads_and(tid != 0 || mbar_wait(&bar[sn], phase[sn])) != 0;
        phase[sn] ^= 1u;
      }
      if (ok) issue(kn, sn);
    }
    cp_async_commit();  // possibly empty: keeps the group count of the wait above uniform
  }
  // the commits not waited for yet: chunks max(kc0, kc1 - S) .. kc1 - 1, each on its own stage
  for (int c = max(kc0, kc1 - S); c < kc1 && ok; ++c) {
    const int st = (c - kc0) % S;
    ok = __syncthreads_and(tid != 0 || mbar_wait(&bar[st], phase[st])) != 0;
    phase[st] ^= 1u;
  }
  cp_async_wait<0>();
  tc_fence_after();
  if (!ok) {
    if (tid == 0) atomicOr(g.err, (unsigned)PCSIR_DERR_TIMEOUT);
  } else {
    gemm_epilogue<NT>(g, tmem, m0, n0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, NCOLS);
}

// ---------------------------------------------------------------------------
// TMA variant (same operand condition): the copy engine brings each K chunk of A and B into a stage
// as two tensor tiles (cp.async.bulk.tensor with 128-byte swizzle, which is exactly the K-major
// layout the MMAs read), completing on the stage's "full" mbarrier with its byte count; one thread
// issues the copies, another the MMAs, which release the stage through its "empty" mbarrier.  No
// block-wide barrier inside the K loop.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

template <int NT, int S>
__global__ void __launch_bounds__(MM_THREADS) k_gemm_bf16_tma(GemmArgs g, const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ __align__(1024) uint8_t mm_smem_raw[];
  uint8_t* mm_smem = align1024(mm_smem_raw);
  constexpr int SA = MM_M * MM_K * 2, SB = NT * MM_K * 2, ST = SA + SB;
  uint64_t* full = reinterpret_cast<uint64_t*>(mm_smem + S * ST);
  uint64_t* empty = full + S;
  uint64_t* done = empty + S;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int s_abort, s_issued, s_used;
  const uint32_t s0 = smem_u32(mm_smem);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * MM_M;
  const int n0 = blockIdx.y * NT;
  const int nk_total = (g.K + MM_K - 1) / MM_K;
  int kc0 = 0, kc1 = nk_total;
  if (g.kchunks_per_split > 0) {
    kc0 = blockIdx.z * g.kchunks_per_split;
    kc1 = min(nk_total, kc0 + g.kchunks_per_split);
  }
  if (kc0 >= kc1) return;  // empty K slice (uniform over the block)
  constexpr uint32_t NCOLS = NT < 32 ? 32 : NT;
  if (warp == 0) tc_alloc(tslot, NCOLS);
  if (tid == 0) {
#pragma unroll
    for (int j = 0; j < S; ++j) {
      mbar_init(&full[j], 1);
      mbar_init(&empty[j], 1);
    }
    mbar_init(done, 1);
    s_abort = 0;
    s_issued = 0;
    s_used = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int nk = kc1 - kc0;
  if (tid == 0) {
    // copies: stage i % S for chunk kc0 + i, after the MMAs of chunk kc0 + i - S released it
    for (int i = 0; i < nk; ++i) {
      const int st = i % S, use = i / S;
      if (use > 0 && !mbar_wait(&empty[st], (uint32_t)((use - 1) & 1))) {
        atomicExch(&s_abort, 1);
        break;
      }
      if (*(volatile int*)&s_abort) break;
      mbar_expect_tx(&full[st], (uint32_t)ST);
      tma_load_2d(s0 + st * ST, &tmA, (kc0 + i) * MM_K, m0, &full[st]);
      tma_load_2d(s0 + st * ST + SA, &tmB, (kc0 + i) * MM_K, n0, &full[st]);
      s_issued = i + 1;
    }
  } else if (tid == 32) {
    // MMAs of chunk kc0 + i once its two tiles have landed; each stage is released by a commit
    const uint32_t idesc = mm_idesc(MM_M, NT);
    for (int i = 0; i < nk; ++i) {
      const int st = i % S, use = i / S;
      if (!mbar_wait(&full[st], (uint32_t)(use & 1))) {
        atomicExch(&s_abort, 1);
        break;
      }
      s_used = i + 1;
      tc_fence_after();
      tc_mma_chunk(tmem, s0 + st * ST, s0 + st * ST + SA, idesc, i == 0);
      tc_commit(&empty[st]);
    }
    tc_commit(done);  // arrives when every MMA issued above has completed
  }
  __syncthreads();
  // the MMA thread always commits to done, so this wait also covers a stopped loop's MMAs
  const bool drained = __syncthreads_and(tid != 0 || mbar_wait(done, 0u)) != 0;
  const bool ok = s_abort == 0 && drained;
  if (!ok && tid == 0) {
    // copies issued but never waited for: let them land (bounded) before the block leaves
    for (int i = s_used; i < s_issued; ++i) mbar_wait(&full[i % S], (uint32_t)((i / S) & 1));
  }
  tc_fence_after();
  if (!ok) {
    if (tid == 0) atomicOr(g.err, (unsigned)PCSIR_DERR_TIMEOUT);
  } else {
    gemm_epilogue<NT>(g, tmem, m0, n0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, NCOLS);
}

constexpr int GEMM_ASYNC_STAGES = 4;
template <int NT>
constexpr int gemm_async_smem() {
  // the stages, the 1024-byte alignment slack, and the barriers and TMEM slot (at most 2 S + 2 words)
  return GEMM_ASYNC_STAGES * (MM_M * MM_K * 2 + NT * MM_K * 2) + 1024 + 128;
}

// 100 KB of dynamic shared memory (more than the 49 KB the 256-column tile
// uses) caps residency at two CTAs per SM, so two tiles of 256 TMEM columns
// always fit.
constexpr int GEMM_SMEM = 100 * 1024;

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// a K-contiguous bf16 operand [rows][K] (row stride ld elements) as 64 x box_rows tiles
bool make_operand_map(CUtensorMap* m, const __nv_bfloat16* base, int K, int rows, long long ld, int box_rows) {
  if (!g_encode) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2u};
  const cuuint32_t box[2] = {(cuuint32_t)MM_K, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

cudaError_t prepare_gemm() {
  static std::once_flag once;
  static cudaError_t status = cudaSuccess;
  std::call_once(once, [] {
    status = cudaFuncSetAttribute(k_gemm_bf16<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
    if (status == cudaSuccess)
      status = cudaFuncSetAttribute(k_gemm_bf16<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
    if (status == cudaSuccess)
      status = cudaFuncSetAttribute(k_gemm_bf16_async<256, GEMM_ASYNC_STAGES>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, gemm_async_smem<256>());
    if (status == cudaSuccess)
      status = cudaFuncSetAttribute(k_gemm_bf16_async<64, GEMM_ASYNC_STAGES>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, gemm_async_smem<64>());
    if (status == cudaSuccess)
      status = cudaFuncSetAttribute(k_gemm_bf16_tma<256, GEMM_ASYNC_STAGES>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, gemm_async_smem<256>());
    if (status == cudaSuccess)
      status = cudaFuncSetAttribute(k_gemm_bf16_tma<64, GEMM_ASYNC_STAGES>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, gemm_async_smem<64>());
    // the tensor-map encoder, from the driver (none: the cp.async path is used)
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  });
  return status;
}

cudaError_t launch_gemm(GemmArgs g, cudaStream_t s, int nt, int splits) {
  if (nt == 0) nt = g.N > 64 ? 256 : 64;
  const int nk = (g.K + MM_K - 1) / MM_K;
  splits = std::max(1, std::min(splits, nk));
  g.kchunks_per_split = 0;
  if (splits > 1) {
    if (g.epi != EPI_ATOMIC) return cudaErrorInvalidValue;
    g.kchunks_per_split = (nk + splits - 1) / splits;
    splits = (nk + g.kchunks_per_split - 1) / g.kchunks_per_split;
  }
  dim3 grid((g.M + MM_M - 1) / MM_M, (g.N + nt - 1) / nt, splits);
  // K-contiguous operands on 16-byte boundaries take the multi-stage path
  const bool async_ok = g.sak == 1 && g.sbk == 1 && (g.sam % 8) == 0 && (g.sbn % 8) == 0 &&
                        ((reinterpret_cast<uintptr_t>(g.A) | reinterpret_cast<uintptr_t>(g.B)) & 15u) == 0u;
  CUtensorMap ma, mb;
  if (async_ok && make_operand_map(&ma, g.A, g.K, g.M, g.sam, MM_M) && make_operand_map(&mb, g.B, g.K, g.N, g.sbn, nt)) {
    if (nt == 256)
      k_gemm_bf16_tma<256, GEMM_ASYNC_STAGES><<<grid, MM_THREADS, gemm_async_smem<256>(), s>>>(g, ma, mb);
    else
      k_gemm_bf16_tma<64, GEMM_ASYNC_STAGES><<<grid, MM_THREADS, gemm_async_smem<64>(), s>>>(g, ma, mb);
  } else if (async_ok) {
    if (nt == 256)
      k_gemm_bf16_async<256, GEMM_ASYNC_STAGES><<<grid, MM_THREADS, gemm_async_smem<256>(), s>>>(g);
    else
      k_gemm_bf16_async<64, GEMM_ASYNC_STAGES><<<grid, MM_THREADS, gemm_async_smem<64>(), s>>>(g);
  } else if (nt == 256) {
    k_gemm_bf16<256><<<grid, MM_THREADS, GEMM_SMEM, s>>>(g);
  } else {
    k_gemm_bf16<64><<<grid, MM_THREADS, GEMM_SMEM, s>>>(g);
  }
  return cudaGetLastError();
}

}  // namespace pcsir

using namespace pcsir;

namespace {
std::mutex g_gemm_mu;
unsigned* g_gemm_err = nullptr;
}  // namespace

extern "C" pcsir_status pcsir_gemm_bf16(const uint16_t* A, int64_t sam, int64_t sak, const uint16_t* B, int64_t sbn,
                                        int64_t sbk, float* C, int64_t ldc, int32_t M, int32_t N, int32_t K,
                                        int32_t accumulate, void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1) return PCSIR_EINVAL;
  {
    std::lock_guard<std::mutex> lock(g_gemm_mu);
    if (prepare_gemm() != cudaSuccess) return PCSIR_ECUDA;
    if (!g_gemm_err) {
      if (cudaMalloc(&g_gemm_err, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        g_gemm_err = nullptr;
        return PCSIR_ENOMEM;
      }
      if (cudaMemset(g_gemm_err, 0, sizeof(unsigned)) != cudaSuccess) return PCSIR_ECUDA;
    }
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
