// Systematic resampling for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc: a host application
// whose device-memory budget is fixed and fully handed out at start-up, a
// framework whose caching allocator already owns the free memory, or a
// real-time tracking loop that must not take the implicit device-wide
// synchronisation an allocation can cause.  pcsir_resample_noalloc gives them
// the resampling step without a context: its scratch (control block, result,
// per-tile sums) lives in a fixed-size array in the library's own device
// memory, so nothing is allocated at any call.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds it (about 17 KB) until the process exits.  Host code cannot
// use the array's name as a device address, so the first call on each device
// (with that device current) looks the address up with cudaGetSymbolAddress
// and caches it; that first call should come before any stream capture.  The
// cache is keyed by the device's current CUDA context: a new primary context
// (after cudaDeviceReset, say) reloads the library's module, so the next call
// looks the address up again instead of using a stale one.  Every call shares
// the one array per device, and the array keeps the last call's contents:
// each call clears the parts that must start at zero, and calls whose work
// overlaps on the GPU race on it.
#include <cuda.h>

#include <mutex>

#include "pcsir_internal.h"

namespace pcsir {

constexpr int64_t NOALLOC_MAX_N = int64_t(1) << 22;  // 4,194,304 particles per call
constexpr int64_t NOALLOC_MAX_TILES = NOALLOC_MAX_N / SCAN_TILE;

struct NoallocScratch {
  Control ctl;
  pcsir_result res;
  long long tile_sum[NOALLOC_MAX_TILES];
  long long tile_excl[NOALLOC_MAX_TILES];
  long long tile_lo[NOALLOC_MAX_TILES + 1];
  int tile_ovx[NOALLOC_MAX_TILES + 1];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};
int g_num_sms[MAX_DEVICES] = {};
unsigned long long g_ctx_id[MAX_DEVICES] = {};  // context the cached address belongs to

// Driver entry points for the current context's unique id, looked up through
// the runtime (the library does not link the driver library directly).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

cudaError_t current_context_id(unsigned long long* id) {
  if (!g_ctx_get_current || !g_ctx_get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorNotSupported;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext c = nullptr;
  if (g_ctx_get_current(&c) != CUDA_SUCCESS || c == nullptr) return cudaErrorDeviceUninitialized;
  if (g_ctx_get_id(c, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

// Once per device and context, with that device current: the scratch array's
// device address, the SM count, and the resampling kernel's shared-memory limit.
cudaError_t setup_current_device(NoallocScratch** scratch, int* num_sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  // make the device's primary context current (initialising it on first use)
  e = cudaSetDevice(dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  unsigned long long id = 0;
  e = current_context_id(&id);
  if (e != cudaSuccess) return e;
  if (g_scratch_ptr[dev] == nullptr || g_ctx_id[dev] != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = prepare_resample();
    if (e != cudaSuccess) return e;
    g_num_sms[dev] = sms;
    g_scratch_ptr[dev] = p;
    g_ctx_id[dev] = id;
  }
  *scratch = static_cast<NoallocScratch*>(g_scratch_ptr[dev]);
  *num_sms = g_num_sms[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace pcsir

using namespace pcsir;

extern "C" pcsir_status pcsir_resample_noalloc(const double* logw, int64_t N, double u0, int32_t* ancestors,
                                               void* stream) {
  if (!logw || !ancestors || N < 1) return PCSIR_EINVAL;
  if (N > NOALLOC_MAX_N) return PCSIR_ERANGE;
  if (!(u0 >= 0.0 && u0 < 1.0)) return PCSIR_EINVAL;
  NoallocScratch* sc = nullptr;
  int num_sms = 0;
  if (setup_current_device(&sc, &num_sms) != cudaSuccess) {
    cudaGetLastError();
    return PCSIR_ECUDA;
  }
  StepBuffers b{};
  b.ctl = &sc->ctl;
  b.dres = &sc->res;
  b.derr_out = &sc->res.device_error;
  b.tile_sum = sc->tile_sum;
  b.tile_excl = sc->tile_excl;
  b.tile_lo = sc->tile_lo;
  b.tile_ovx = sc->tile_ovx;
  b.max_tiles = NOALLOC_MAX_TILES;
  b.hbits = 10;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(&sc->ctl, 0, sizeof(Control), s);
  if (e == cudaSuccess) e = launch_logw_front(b, logw, N, num_sms, s);
  if (e == cudaSuccess) e = launch_resample_logw(b, logw, ancestors, N, u0, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PCSIR_ECUDA;
  }
  return PCSIR_OK;
}
