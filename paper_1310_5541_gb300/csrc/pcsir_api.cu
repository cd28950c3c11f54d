// Host side of the C ABI declared in include/pcsir.h: context lifetime,
// argument checks, workspace, and the kernel sequence of one filter step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pcsir_internal.h"
#include "pcsir_philox.cuh"

using namespace pcsir;

struct pcsir_ctx {
  pcsir_config cfg{};
  int device = 0;
  int num_sms = 0;
  StepBuffers b{};
  ModelParams m{};
  pcsir_result* host_res = nullptr;  // page-locked copy of the last result
  std::vector<void*> allocs;
  std::string err = "no error";
  bool failed = false;
  int last_kind = -1;
  int64_t last_N = 0;
  // attached likelihood surrogate: per-step held-out list and statistics
  SurStep sur{};
  bool sur_on = false;
  bool sur_ran = false;          // the last pcSIR step used the surrogate
  unsigned long long sur_steps = 0;
  // deferred resampling run: the particle set is b.prop[., def_anc[i]] (def_has_anc) or b.prop
  void* def_other = nullptr;  // the run's second state buffer
  int32_t* def_anc = nullptr;
  bool def_active = false;
  bool def_has_anc = false;
  bool last_deferred = false;  // the last step was a deferred one (its ancestors are def_anc)
  int64_t def_N = 0;
  // stage timing: 5 events per step slot
  std::vector<cudaEvent_t> events;
  int timing_slots = 0;
  int64_t timing_count = 0;  // steps recorded since enable / last read
};

namespace {

pcsir_status fail(pcsir_ctx* c, pcsir_status st, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (st == PCSIR_ECUDA) c->failed = true;
  }
  return st;
}

pcsir_status cuda_fail(pcsir_ctx* c, cudaError_t e, const char* what) {
  return fail(c, PCSIR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
bool dev_alloc(pcsir_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return true;
}

void free_events(pcsir_ctx* c) {
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  c->events.clear();
  c->timing_slots = 0;
  c->timing_count = 0;
}

// events of the step about to be enqueued (nullptr when timing is off)
StageEvents step_events(pcsir_ctx* c) {
  if (c->timing_slots == 0) return StageEvents{nullptr};
  const int slot = (int)(c->timing_count % c->timing_slots);
  c->timing_count++;
  return StageEvents{c->events.data() + 5 * slot};
}

void free_all(pcsir_ctx* c) {
  free_events(c);
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->host_res) cudaFreeHost(c->host_res);
  c->host_res = nullptr;
}

size_t state_size(const pcsir_ctx* c) { return c->cfg.state_dtype == PCSIR_F64 ? 8 : 4; }

pcsir_status check_step_args(pcsir_ctx* c, const void* state, int64_t N, const float* image, int32_t W, int32_t H,
                             const void* noise, double u0) {
  if (!c) return PCSIR_EINVAL;
  if (c->failed) return fail(c, PCSIR_ESTATE, "context failed earlier: " + c->err);
  if (!state || !image) return fail(c, PCSIR_EINVAL, "state and image must be non-NULL device pointers");
  if (!noise) return fail(c, PCSIR_ENOTSUP, "noise must be a device array; in-kernel noise is not supported");
  if (N < 1) return fail(c, PCSIR_EINVAL, "N must be >= 1");
  if (N > c->cfg.max_particles) return fail(c, PCSIR_ERANGE, "N exceeds max_particles of the context");
  if (W < 1 || H < 1) return fail(c, PCSIR_EINVAL, "image width and height must be >= 1");
  if (!(u0 >= 0.0 && u0 < 1.0)) return fail(c, PCSIR_EINVAL, "u0 must lie in [0, 1)");
  return PCSIR_OK;
}

// a plain step overwrites the propagated-state buffer a deferred run keeps its particles in
void end_deferred(pcsir_ctx* c) {
  c->def_active = false;
  c->last_deferred = false;
}

pcsir_status finish_step(pcsir_ctx* c, cudaStream_t s, pcsir_result* result_host, int kind, int64_t N) {
  cudaError_t e = cudaMemcpyAsync(c->host_res, c->b.dres, sizeof(pcsir_result), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy of step result");
  if (result_host && result_host != c->host_res) {
    e = cudaMemcpyAsync(result_host, c->b.dres, sizeof(pcsir_result), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy of step result");
  }
  c->last_kind = kind;
  c->last_N = N;
  return PCSIR_OK;
}

}  // namespace

extern "C" {

const char* pcsir_version(void) { return "pcsir-gb300 0.1 (sm_103a)"; }

const char* pcsir_last_error(pcsir_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

pcsir_status pcsir_create(const pcsir_config* cfg, pcsir_ctx** out) {
  if (!out) return PCSIR_EINVAL;
  *out = nullptr;
  if (!cfg) return PCSIR_EINVAL;
  if (cfg->state_dtype != PCSIR_F32 && cfg->state_dtype != PCSIR_F64) return PCSIR_EINVAL;
  if (cfg->lik_kind != PCSIR_LIK_POISSON && cfg->lik_kind != PCSIR_LIK_SSE) return PCSIR_EINVAL;
  if (cfg->patch < 1 || cfg->patch > 127 || (cfg->patch & 1) == 0) return PCSIR_EINVAL;
  if (!(cfg->psf_sigma > 0.0) || !std::isfinite(cfg->psf_sigma)) return PCSIR_EINVAL;
  if (cfg->lik_kind == PCSIR_LIK_POISSON && !(cfg->bg > 0.0)) return PCSIR_EINVAL;
  if (cfg->lik_kind == PCSIR_LIK_SSE && !(cfg->sigma_xi > 0.0)) return PCSIR_EINVAL;
  if (!std::isfinite(cfg->bg)) return PCSIR_EINVAL;
  if (cfg->max_particles < 1 || cfg->max_particles > MAX_PARTICLES) return PCSIR_EINVAL;
  if (cfg->keep & ~(PCSIR_KEEP_ANCESTORS | PCSIR_KEEP_WEIGHTS | PCSIR_KEEP_PARTICLE_BIN | PCSIR_KEEP_LOGLIK |
                    PCSIR_KEEP_QWEIGHTS))
    return PCSIR_EINVAL;
  if ((cfg->dummy != PCSIR_DUMMY_COM && cfg->dummy != PCSIR_DUMMY_COC) || cfg->reserved != 0) return PCSIR_EINVAL;

  pcsir_ctx* c = new (std::nothrow) pcsir_ctx();
  if (!c) return PCSIR_ENOMEM;
  c->cfg = *cfg;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    cudaGetLastError();
    return PCSIR_ECUDA;
  }
  c->m.P = cfg->patch;
  c->m.kind = cfg->lik_kind;
  c->m.sigma = cfg->psf_sigma;
  c->m.bg = cfg->bg;
  c->m.sigma_xi = cfg->sigma_xi > 0.0 ? cfg->sigma_xi : 1.0;
  c->m.coc = cfg->dummy == PCSIR_DUMMY_COC ? 1 : 0;

  const int64_t nmax = cfg->max_particles;
  int hbits = 1;
  while ((int64_t(1) << hbits) < 2 * nmax) ++hbits;
  if (hbits < 10) hbits = 10;
  const size_t hcap = size_t(1) << hbits;
  StepBuffers& b = c->b;
  b.hbits = hbits;
  b.bin_stride = nmax;
  b.max_tiles = (nmax + SCAN_TILE - 1) / SCAN_TILE;
  bool ok = dev_alloc(c, &b.hkey, hcap) && dev_alloc(c, &b.hcnt, hcap) && dev_alloc(c, &b.hsum, 5 * hcap) &&
            dev_alloc(c, &b.hrank, hcap) && dev_alloc(c, &b.hq, hcap) && dev_alloc(c, &b.hw, hcap) &&
            dev_alloc(c, &b.occ, (size_t)nmax) && dev_alloc(c, &b.bin_xy, 2 * (size_t)nmax) &&
            dev_alloc(c, &b.bin_cnt, (size_t)nmax) && dev_alloc(c, &b.dummy, 5 * (size_t)nmax) &&
            dev_alloc(c, &b.bin_ll, (size_t)nmax) && dev_alloc(c, &b.pslot, (size_t)nmax) &&
            dev_alloc(c, &b.llq, (size_t)nmax) && dev_alloc(c, &b.tile_sum, (size_t)b.max_tiles) &&
            dev_alloc(c, &b.tile_excl, (size_t)b.max_tiles) && dev_alloc(c, &b.tile_lo, (size_t)b.max_tiles + 1) &&
            dev_alloc(c, &b.tile_ovx, (size_t)b.max_tiles + 1) &&
            dev_alloc(c, &b.ctl, 1) && dev_alloc(c, &b.dres, 1);
  if (ok) {
    unsigned char* p = nullptr;
    ok = dev_alloc(c, &p, 5 * (size_t)nmax * state_size(c));
    b.prop = p;
  }
  if (ok && (cfg->keep & PCSIR_KEEP_ANCESTORS)) ok = dev_alloc(c, &b.anc, (size_t)nmax);
  if (ok && (cfg->keep & PCSIR_KEEP_WEIGHTS)) ok = dev_alloc(c, &b.wout, (size_t)nmax);
  if (ok && (cfg->keep & PCSIR_KEEP_QWEIGHTS)) ok = dev_alloc(c, &b.qout, (size_t)nmax);
  if (ok && (cfg->keep & PCSIR_KEEP_PARTICLE_BIN)) ok = dev_alloc(c, &b.pbin, (size_t)nmax);
  if (ok && (cfg->keep & PCSIR_KEEP_LOGLIK)) ok = dev_alloc(c, &b.ll, (size_t)nmax);
  if (!ok) {
    free_all(c);
    delete c;
    return PCSIR_ENOMEM;
  }
  b.derr_out = &b.dres->device_error;
  b.resampled_out = &b.dres->resampled;
  e = prepare_kernels(cfg->state_dtype, b.prop_bin_per_sm);
  if (e == cudaSuccess) e = prepare_resample();
  if (e == cudaSuccess) e = cudaMallocHost(&c->host_res, sizeof(pcsir_result));
  if (e == cudaSuccess) e = cudaMemset(b.hkey, 0xff, hcap * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(b.hcnt, 0, hcap * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(b.hsum, 0, 5 * hcap * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(b.dres, 0, sizeof(pcsir_result));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return e == cudaErrorMemoryAllocation ? PCSIR_ENOMEM : PCSIR_ECUDA;
  }
  std::memset(c->host_res, 0, sizeof(pcsir_result));
  *out = c;
  return PCSIR_OK;
}

pcsir_status pcsir_destroy(pcsir_ctx* ctx) {
  if (!ctx) return PCSIR_OK;
  cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
  return PCSIR_OK;
}

namespace {

// checks of the generator's arguments: FP32 state, finite non-negative deviations, a 32-bit frame
pcsir_status make_noise_gen(pcsir_ctx* ctx, const double* q, uint64_t seed, uint64_t frame, NoiseGen* ng) {
  if (ctx->cfg.state_dtype != PCSIR_F32) return fail(ctx, PCSIR_ENOTSUP, "drawn noise needs FP32 state");
  if (!q) return fail(ctx, PCSIR_EINVAL, "q must point to five standard deviations");
  if (frame > 0xFFFFFFFFull) return fail(ctx, PCSIR_EINVAL, "frame must be below 2^32");
  for (int d = 0; d < 5; ++d)
    if (!(q[d] >= 0.0) || !std::isfinite(q[d])) return fail(ctx, PCSIR_EINVAL, "q must be finite and >= 0");
  ng->seed = seed;
  ng->frame = (unsigned)frame;
  for (int d = 0; d < 5; ++d) ng->q[d] = (float)q[d];
  return PCSIR_OK;
}

pcsir_status step_impl(pcsir_ctx* ctx, void* state, int64_t N, const float* image, int32_t W, int32_t H, double h,
                       const void* noise, const NoiseGen* ng, double u0, void* stream, pcsir_result* result_host) {
  if (!(h > 0.0 && h <= MAX_H)) return fail(ctx, PCSIR_EINVAL, "h must lie in (0, 8]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const StageEvents se = step_events(ctx);
  cudaError_t e = cudaMemsetAsync(ctx->b.ctl, 0, sizeof(Control), s);
  if (e == cudaSuccess && se.ev) e = cudaEventRecord(se.ev[0], s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reset of step control block");
  // Cell-table size of the propagate/bin kernel (results do not depend on it):
  // the large table once the previous step found more cells than the small
  // table holds comfortably, else from the cell size alone.  The previous
  // count is read from the page-locked result copy of that step.
  const int64_t prev_bins = ctx->last_kind == 1 ? ((volatile pcsir_result*)ctx->host_res)->n_bins : -1;
  ctx->b.big_table = prev_bins >= 0 ? (prev_bins > 1200 ? 1 : 0) : (h < 0.15 ? 1 : 0);
  SurStep sp{};
  if (ctx->sur_on && (int64_t)W * H > sur_max_pixels(ctx->sur.sur))
    return fail(ctx, PCSIR_ERANGE, "image larger than the surrogate's max_pixels");
  if (ctx->sur_on) {
    sp = ctx->sur;
    sp.salt = ctx->sur_steps;
    e = cudaMemsetAsync(sp.stats, 0, sizeof(SurStats), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reset of surrogate statistics");
  }
  e = launch_pcsir_front(ctx->b, ctx->m, ctx->cfg.state_dtype, state, noise, N, h, image, W, H, ctx->num_sms, s,
                         se, ctx->sur_on ? &sp : nullptr, nullptr, ng);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pcSIR front kernels");
  if (ctx->sur_on) ctx->sur_steps++;
  ctx->sur_ran = ctx->sur_on;
  e = launch_resample(ctx->b, ctx->cfg.state_dtype, state, N, u0, WSRC_BINS, ctx->cfg.keep, ctx->num_sms, s);
  if (e == cudaSuccess && se.ev) e = cudaEventRecord(se.ev[4], s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan/resample kernel");
  return finish_step(ctx, s, result_host, 1, N);
}

}  // namespace

pcsir_status pcsir_step(pcsir_ctx* ctx, void* state, int64_t N, const float* image, int32_t W, int32_t H, double h,
                        const void* noise, double u0, void* stream, pcsir_result* result_host) {
  pcsir_status st = check_step_args(ctx, state, N, image, W, H, noise, u0);
  if (st != PCSIR_OK) return st;
  end_deferred(ctx);
  return step_impl(ctx, state, N, image, W, H, h, noise, nullptr, u0, stream, result_host);
}

pcsir_status pcsir_step_philox(pcsir_ctx* ctx, void* state, int64_t N, const float* image, int32_t W, int32_t H,
                               double h, const double* q, uint64_t seed, uint64_t frame, double u0, void* stream,
                               pcsir_result* result_host) {
  // the noise argument of the common checks stands for the generator (non-NULL)
  pcsir_status st = check_step_args(ctx, state, N, image, W, H, state, u0);
  if (st != PCSIR_OK) return st;
  NoiseGen ng{};
  if ((st = make_noise_gen(ctx, q, seed, frame, &ng)) != PCSIR_OK) return st;
  end_deferred(ctx);
  return step_impl(ctx, state, N, image, W, H, h, nullptr, &ng, u0, stream, result_host);
}

pcsir_status pcsir_deferred_begin(pcsir_ctx* ctx, const void* state, int64_t N, void* stream) {
  if (!ctx) return PCSIR_EINVAL;
  if (ctx->failed) return fail(ctx, PCSIR_ESTATE, "context failed earlier: " + ctx->err);
  if (!state) return fail(ctx, PCSIR_EINVAL, "state must be a non-NULL device pointer");
  if (N < 1) return fail(ctx, PCSIR_EINVAL, "N must be >= 1");
  if (N > ctx->cfg.max_particles) return fail(ctx, PCSIR_ERANGE, "N exceeds max_particles of the context");
  if (ctx->sur_on) return fail(ctx, PCSIR_ENOTSUP, "deferred resampling does not use the likelihood surrogate");
  end_deferred(ctx);
  const int64_t nmax = ctx->cfg.max_particles;
  if (!ctx->def_other) {
    unsigned char* p = nullptr;
    if (!dev_alloc(ctx, &p, 5 * (size_t)nmax * state_size(ctx)))
      return fail(ctx, PCSIR_ENOMEM, "state buffer of the deferred run");
    ctx->def_other = p;
  }
  if (!ctx->def_anc && !dev_alloc(ctx, &ctx->def_anc, (size_t)nmax))
    return fail(ctx, PCSIR_ENOMEM, "ancestor array of the deferred run");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e =
      cudaMemcpyAsync(ctx->b.prop, state, 5 * (size_t)N * state_size(ctx), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy of the run's initial states");
  ctx->def_active = true;
  ctx->def_has_anc = false;
  ctx->def_N = N;
  return PCSIR_OK;
}

namespace {

pcsir_status deferred_step_impl(pcsir_ctx* ctx, const float* image, int32_t W, int32_t H, double h, const void* noise,
                                const NoiseGen* ng, double u0, void* stream, pcsir_result* result_host) {
  const int64_t N = ctx->def_N;
  pcsir_status st;
  if (!(h > 0.0 && h <= MAX_H)) return fail(ctx, PCSIR_EINVAL, "h must lie in (0, 8]");
  if (ctx->sur_on) return fail(ctx, PCSIR_ENOTSUP, "deferred resampling does not use the likelihood surrogate");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const StageEvents se = step_events(ctx);
  cudaError_t e = cudaMemsetAsync(ctx->b.ctl, 0, sizeof(Control), s);
  if (e == cudaSuccess && se.ev) e = cudaEventRecord(se.ev[0], s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reset of step control block");
  const int64_t prev_bins = ctx->last_kind == 1 ? ((volatile pcsir_result*)ctx->host_res)->n_bins : -1;
  ctx->b.big_table = prev_bins >= 0 ? (prev_bins > 1200 ? 1 : 0) : (h < 0.15 ? 1 : 0);
  // this step reads the run's particles from src (through the last step's ancestors) and
  // propagates them into dst; its resampling records the ancestors only
  void* src = ctx->b.prop;
  void* dst = ctx->def_other;
  StepBuffers b = ctx->b;
  b.prop = dst;
  b.anc = ctx->def_anc;
  e = launch_pcsir_front(b, ctx->m, ctx->cfg.state_dtype, src, noise, N, h, image, W, H, ctx->num_sms, s, se,
                         nullptr, ctx->def_has_anc ? ctx->def_anc : nullptr, ng);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pcSIR front kernels (deferred)");
  e = launch_resample(b, ctx->cfg.state_dtype, nullptr, N, u0, WSRC_BINS, ctx->cfg.keep | PCSIR_KEEP_ANCESTORS,
                      ctx->num_sms, s);
  if (e == cudaSuccess && se.ev) e = cudaEventRecord(se.ev[4], s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan/resample kernel (deferred)");
  ctx->b.prop = dst;
  ctx->def_other = src;
  ctx->def_has_anc = true;
  ctx->sur_ran = false;
  st = finish_step(ctx, s, result_host, 1, N);
  ctx->last_deferred = true;
  return st;
}

}  // namespace

pcsir_status pcsir_deferred_step(pcsir_ctx* ctx, const float* image, int32_t W, int32_t H, double h,
                                 const void* noise, double u0, void* stream, pcsir_result* result_host) {
  if (!ctx) return PCSIR_EINVAL;
  if (!ctx->def_active && !ctx->failed) return fail(ctx, PCSIR_ESTATE, "no deferred run: call pcsir_deferred_begin");
  pcsir_status st = check_step_args(ctx, ctx->b.prop, ctx->def_N, image, W, H, noise, u0);
  if (st != PCSIR_OK) return st;
  return deferred_step_impl(ctx, image, W, H, h, noise, nullptr, u0, stream, result_host);
}

pcsir_status pcsir_deferred_step_philox(pcsir_ctx* ctx, const float* image, int32_t W, int32_t H, double h,
                                        const double* q, uint64_t seed, uint64_t frame, double u0, void* stream,
                                        pcsir_result* result_host) {
  if (!ctx) return PCSIR_EINVAL;
  if (!ctx->def_active && !ctx->failed) return fail(ctx, PCSIR_ESTATE, "no deferred run: call pcsir_deferred_begin");
  pcsir_status st = check_step_args(ctx, ctx->b.prop, ctx->def_N, image, W, H, ctx->b.prop, u0);
  if (st != PCSIR_OK) return st;
  NoiseGen ng{};
  if ((st = make_noise_gen(ctx, q, seed, frame, &ng)) != PCSIR_OK) return st;
  return deferred_step_impl(ctx, image, W, H, h, nullptr, &ng, u0, stream, result_host);
}

pcsir_status pcsir_deferred_state(pcsir_ctx* ctx, void* state, void* stream) {
  if (!ctx) return PCSIR_EINVAL;
  if (ctx->failed) return fail(ctx, PCSIR_ESTATE, "context failed earlier: " + ctx->err);
  if (!ctx->def_active) return fail(ctx, PCSIR_ESTATE, "no deferred run: call pcsir_deferred_begin");
  if (!state) return fail(ctx, PCSIR_EINVAL, "state must be a non-NULL device pointer");
  const cudaError_t e = launch_gather_state(ctx->cfg.state_dtype, ctx->b.prop,
                                            ctx->def_has_anc ? ctx->def_anc : nullptr, state, ctx->def_N,
                                            static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "gather of the run's states");
  return PCSIR_OK;
}

pcsir_status sir_step(pcsir_ctx* ctx, void* state, int64_t N, const float* image, int32_t W, int32_t H,
                      const void* noise, double u0, void* stream, pcsir_result* result_host) {
  pcsir_status st = check_step_args(ctx, state, N, image, W, H, noise, u0);
  if (st != PCSIR_OK) return st;
  end_deferred(ctx);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const StageEvents se = step_events(ctx);
  cudaError_t e = cudaMemsetAsync(ctx->b.ctl, 0, sizeof(Control), s);
  if (e == cudaSuccess && se.ev) e = cudaEventRecord(se.ev[0], s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reset of step control block");
  e = launch_sir_front(ctx->b, ctx->m, ctx->cfg.state_dtype, state, noise, N, image, W, H, ctx->num_sms, s, se,
                       ctx->cfg.keep);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "SIR front kernels");
  e = launch_resample(ctx->b, ctx->cfg.state_dtype, state, N, u0, WSRC_PARTICLES,
                      ctx->cfg.keep & ~PCSIR_KEEP_PARTICLE_BIN, ctx->num_sms, s);
  if (e == cudaSuccess && se.ev) e = cudaEventRecord(se.ev[4], s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan/resample kernel");
  return finish_step(ctx, s, result_host, 0, N);
}

namespace {
// arguments shared by the two ESS-thresholded steps
pcsir_status check_ess_args(pcsir_ctx* ctx, const int64_t* logw, double ess_min) {
  if (!logw) return fail(ctx, PCSIR_EINVAL, "logw must be a non-NULL device pointer");
  if (ess_min != ess_min) return fail(ctx, PCSIR_EINVAL, "ess_min must not be NaN");
  if (ctx->cfg.state_dtype != PCSIR_F32) return fail(ctx, PCSIR_ENOTSUP, "ESS-thresholded steps take FP32 state");
  if (ctx->sur_on) return fail(ctx, PCSIR_ENOTSUP, "ESS-thresholded steps do not use the likelihood surrogate");
  return PCSIR_OK;
}
}  // namespace

pcsir_status pcsir_step_ess(pcsir_ctx* ctx, void* state, int64_t* logw, int64_t N, const float* image, int32_t W,
                            int32_t H, double h, const void* noise, double u0, double ess_min, void* stream,
                            pcsir_result* result_host) {
  pcsir_status st = check_step_args(ctx, state, N, image, W, H, noise, u0);
  if (st != PCSIR_OK) return st;
  end_deferred(ctx);
  if ((st = check_ess_args(ctx, logw, ess_min)) != PCSIR_OK) return st;
  if (!(h > 0.0 && h <= MAX_H)) return fail(ctx, PCSIR_EINVAL, "h must lie in (0, 8]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(ctx->b.ctl, 0, sizeof(Control), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reset of step control block");
  const int64_t prev_bins = ctx->last_kind == 1 ? ((volatile pcsir_result*)ctx->host_res)->n_bins : -1;
  ctx->b.big_table = prev_bins >= 0 ? (prev_bins > 1200 ? 1 : 0) : (h < 0.15 ? 1 : 0);
  StepBuffers b = ctx->b;
  b.lw_out = reinterpret_cast<long long*>(logw);
  b.ess_min = ess_min;
  const long long* lw_in = reinterpret_cast<const long long*>(logw);
  e = launch_prop_bin(b, PCSIR_F32, state, noise, N, h, ctx->num_sms, s);
  if (e == cudaSuccess) e = launch_pcsir_ess_front(b, ctx->m, lw_in, image, W, H, N, h, ctx->num_sms, s);
  if (e == cudaSuccess) e = launch_particle_weights(b, PCSIR_F32, N, ctx->num_sms, 2, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pcSIR front kernels (ESS)");
  e = launch_resample(b, PCSIR_F32, state, N, u0, WSRC_Q, ctx->cfg.keep, ctx->num_sms, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan/resample kernel");
  return finish_step(ctx, s, result_host, 1, N);
}

pcsir_status sir_step_ess(pcsir_ctx* ctx, void* state, int64_t* logw, int64_t N, const float* image, int32_t W,
                          int32_t H, const void* noise, double u0, double ess_min, void* stream,
                          pcsir_result* result_host) {
  pcsir_status st = check_step_args(ctx, state, N, image, W, H, noise, u0);
  if (st != PCSIR_OK) return st;
  end_deferred(ctx);
  if ((st = check_ess_args(ctx, logw, ess_min)) != PCSIR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(ctx->b.ctl, 0, sizeof(Control), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reset of step control block");
  StepBuffers b = ctx->b;
  b.lw_out = reinterpret_cast<long long*>(logw);
  b.ess_min = ess_min;
  const StageEvents none{};
  e = launch_sir_front(b, ctx->m, PCSIR_F32, state, noise, N, image, W, H, ctx->num_sms, s, none, ctx->cfg.keep,
                       0);
  if (e == cudaSuccess) e = launch_sir_ess_front(b, reinterpret_cast<const long long*>(logw), N, ctx->num_sms, s);
  if (e == cudaSuccess) e = launch_particle_weights(b, PCSIR_F32, N, ctx->num_sms, 0, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "SIR front kernels (ESS)");
  e = launch_resample(b, PCSIR_F32, state, N, u0, WSRC_Q, ctx->cfg.keep & ~PCSIR_KEEP_PARTICLE_BIN,
                      ctx->num_sms, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan/resample kernel");
  return finish_step(ctx, s, result_host, 0, N);
}

pcsir_status pcsir_loglik(pcsir_ctx* ctx, const double* x, const double* y, const double* I0, int64_t n,
                          const float* image, int32_t W, int32_t H, double* out, void* stream) {
  if (!ctx) return PCSIR_EINVAL;
  if (ctx->failed) return fail(ctx, PCSIR_ESTATE, "context failed earlier: " + ctx->err);
  if (n < 0) return fail(ctx, PCSIR_EINVAL, "n must be >= 0");
  if (n == 0) return PCSIR_OK;
  if (!x || !y || !I0 || !image || !out) return fail(ctx, PCSIR_EINVAL, "NULL device pointer");
  if (W < 1 || H < 1) return fail(ctx, PCSIR_EINVAL, "image width and height must be >= 1");
  cudaError_t e = launch_loglik(ctx->m, x, y, I0, n, image, W, H, out, ctx->num_sms, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "likelihood kernel");
  return PCSIR_OK;
}

pcsir_status pcsir_resample(pcsir_ctx* ctx, const double* logw, int64_t N, double u0, int32_t* ancestors,
                            void* stream) {
  if (!ctx) return PCSIR_EINVAL;
  if (ctx->failed) return fail(ctx, PCSIR_ESTATE, "context failed earlier: " + ctx->err);
  if (!logw || !ancestors) return fail(ctx, PCSIR_EINVAL, "NULL device pointer");
  if (N < 1) return fail(ctx, PCSIR_EINVAL, "N must be >= 1");
  if (N > ctx->cfg.max_particles) return fail(ctx, PCSIR_ERANGE, "N exceeds max_particles of the context");
  if (!(u0 >= 0.0 && u0 < 1.0)) return fail(ctx, PCSIR_EINVAL, "u0 must lie in [0, 1)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(ctx->b.ctl, 0, sizeof(Control), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reset of step control block");
  e = launch_logw_front(ctx->b, logw, N, ctx->num_sms, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "weight reduction");
  e = launch_resample_logw(ctx->b, logw, ancestors, N, u0, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan/resample kernel");
  ctx->last_kind = -1;
  return PCSIR_OK;
}

pcsir_status pcsir_timing_enable(pcsir_ctx* ctx, int32_t max_steps) {
  if (!ctx || max_steps < 0 || max_steps > 100000) return PCSIR_EINVAL;
  if (ctx->failed) return fail(ctx, PCSIR_ESTATE, "context failed earlier: " + ctx->err);
  free_events(ctx);
  if (max_steps == 0) return PCSIR_OK;
  ctx->events.resize(5 * (size_t)max_steps, nullptr);
  for (auto& ev : ctx->events) {
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
      ev = nullptr;
      free_events(ctx);
      return cuda_fail(ctx, e, "event creation");
    }
  }
  ctx->timing_slots = max_steps;
  ctx->timing_count = 0;
  return PCSIR_OK;
}

pcsir_status pcsir_timing_read(pcsir_ctx* ctx, float* ms, int32_t capacity, int32_t* n_steps) {
  if (!ctx || !ms || !n_steps || capacity < 0) return PCSIR_EINVAL;
  if (ctx->timing_slots == 0) return fail(ctx, PCSIR_ESTATE, "timing is not enabled");
  const int64_t n = ctx->timing_count < ctx->timing_slots ? ctx->timing_count : ctx->timing_slots;
  const int64_t first = ctx->timing_count - n;
  int32_t written = 0;
  for (int64_t k = 0; k < n && 4 * (written + 1) <= capacity; ++k) {
    const int slot = (int)((first + k) % ctx->timing_slots);
    cudaEvent_t* ev = ctx->events.data() + 5 * slot;
    cudaError_t e = cudaEventSynchronize(ev[4]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event synchronisation");
    for (int j = 0; j < 4; ++j) {
      float t = 0.0f;
      e = cudaEventElapsedTime(&t, ev[j], ev[j + 1]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "event elapsed time");
      ms[4 * written + j] = t;
    }
    ++written;
  }
  *n_steps = written;
  ctx->timing_count = 0;
  return PCSIR_OK;
}

pcsir_status pcsir_get_outputs(pcsir_ctx* ctx, pcsir_outputs* o) {
  if (!ctx || !o) return PCSIR_EINVAL;
  if (ctx->last_kind < 0) return fail(ctx, PCSIR_ESTATE, "no step has run on this context");
  std::memset(o, 0, sizeof(*o));
  const StepBuffers& b = ctx->b;
  o->n_particles = ctx->last_N;
  o->n_bins = ctx->last_kind == 1 ? ctx->host_res->n_bins : 0;
  o->bin_stride = b.bin_stride;
  o->prop_state = b.prop;
  if (ctx->last_kind == 1) {
    o->bin_xy = b.bin_xy;
    o->bin_count = b.bin_cnt;
    o->dummy = b.dummy;
    o->bin_loglik = b.bin_ll;
    o->particle_bin = b.pbin;
  } else {
    o->loglik = b.ll;
  }
  o->ancestor = ctx->last_deferred ? ctx->def_anc : b.anc;
  o->weight = b.wout;
  o->qweight = reinterpret_cast<const int64_t*>(b.qout);
  return PCSIR_OK;
}

pcsir_status pcsir_attach_surrogate(pcsir_ctx* ctx, pcsir_surrogate* sur, double holdout_frac, int32_t min_holdout,
                                    double window, double max_err) {
  if (!ctx) return PCSIR_EINVAL;
  if (ctx->failed) return fail(ctx, PCSIR_ESTATE, "context failed earlier: " + ctx->err);
  if (!sur) {
    ctx->sur_on = false;
    return PCSIR_OK;
  }
  if (!(holdout_frac >= 0.0 && holdout_frac <= 1.0) || min_holdout < 0 || !(window >= 0.0) || !(max_err >= 0.0))
    return fail(ctx, PCSIR_EINVAL, "invalid held-out fraction, window or error threshold");
  if (ctx->cfg.patch != PCSIR_SUR_PATCH || ctx->cfg.lik_kind != PCSIR_LIK_POISSON)
    return fail(ctx, PCSIR_EINVAL, "the surrogate models the Poisson likelihood over a 21 x 21 patch");
  if (sur_dim(sur) != 2) return fail(ctx, PCSIR_EINVAL, "a 3D surrogate attaches to a 3D context");
  SurStep& sp = ctx->sur;
  if (!sp.stats) {
    constexpr int HO_CAP = 1 << 16;
    if (!(dev_alloc(ctx, &sp.ho_bin, HO_CAP) && dev_alloc(ctx, &sp.ho_ll, HO_CAP) && dev_alloc(ctx, &sp.stats, 1))) {
      sp.stats = nullptr;
      return fail(ctx, PCSIR_ENOMEM, "held-out list allocation");
    }
    sp.ho_cap = HO_CAP;
    cudaError_t e = cudaMemset(sp.stats, 0, sizeof(SurStats));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "held-out statistics");
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

// ---------------------------------------------------------------------------
// Checkpoint and resume.  File layout (host byte order), each record fixed size:
//   char magic[8] = "PCSIRCK1"; uint32 version = 1; uint32 flags (bit 0: surrogate record)
//   pcsir_config cfg
//   uint64 held-out salt (surrogate-assisted steps since the attach); double holdout_frac,
//   window, max_err; int32 min_holdout, int32 0
//   [flags & 1] double i0_ref, sigma_ref, label_mean, label_scale; float params[NPARAMS]
//   uint64 FNV-1a hash of every byte before it
// ---------------------------------------------------------------------------
namespace {

constexpr char CK_MAGIC[8] = {'P', 'C', 'S', 'I', 'R', 'C', 'K', '1'};
constexpr uint32_t CK_VERSION = 1;

struct CkHead {
  char magic[8];
  uint32_t version;
  uint32_t flags;
  pcsir_config cfg;
  uint64_t salt;
  double frac, window, max_err;
  int32_t min_holdout, pad;
};

struct CkSur {
  double i0_ref, sigma_ref, label_mean, label_scale;
};

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}
constexpr uint64_t FNV_OFFSET = 14695981039346656037ull;

// configs that give the same steps: every field but the kept outputs
bool same_model(const pcsir_config& a, const pcsir_config& b) {
  return a.state_dtype == b.state_dtype && a.lik_kind == b.lik_kind && a.patch == b.patch &&
         a.psf_sigma == b.psf_sigma && a.bg == b.bg && a.sigma_xi == b.sigma_xi && a.dummy == b.dummy;
}

}  // namespace

pcsir_status pcsir_save(pcsir_ctx* ctx, const char* path) {
  if (!ctx || !path) return PCSIR_EINVAL;
  if (ctx->failed) return fail(ctx, PCSIR_ESTATE, "context failed earlier: " + ctx->err);
  CkHead h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, CK_MAGIC, sizeof(CK_MAGIC));
  h.version = CK_VERSION;
  h.flags = ctx->sur_on ? 1u : 0u;
  h.cfg = ctx->cfg;
  h.salt = ctx->sur_steps;
  h.frac = ctx->sur.frac;
  h.window = ctx->sur.window;
  h.max_err = ctx->sur.max_err;
  h.min_holdout = ctx->sur.min_holdout;
  std::vector<float> params;
  CkSur sr{};
  if (ctx->sur_on) {
    params.resize(PCSIR_SUR_NPARAMS);
    pcsir_surrogate* sur = const_cast<pcsir_surrogate*>(ctx->sur.sur);
    const pcsir_status st = pcsir_surrogate_get_params(sur, params.data(), &sr.label_mean, &sr.label_scale);
    if (st != PCSIR_OK) return fail(ctx, st, "reading the attached surrogate's parameters");
    sur_refs(sur, &sr.i0_ref, &sr.sigma_ref);
  }
  uint64_t hash = fnv1a(FNV_OFFSET, &h, sizeof(h));
  if (ctx->sur_on) {
    hash = fnv1a(hash, &sr, sizeof(sr));
    hash = fnv1a(hash, params.data(), params.size() * sizeof(float));
  }
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(ctx, PCSIR_EINVAL, std::string("cannot open ") + tmp + " for writing");
  bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
  if (ok && ctx->sur_on)
    ok = std::fwrite(&sr, sizeof(sr), 1, f) == 1 &&
         std::fwrite(params.data(), sizeof(float), params.size(), f) == params.size();
  ok = ok && std::fwrite(&hash, sizeof(hash), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(ctx, PCSIR_EINVAL, std::string("cannot write checkpoint ") + path);
  }
  return PCSIR_OK;
}

pcsir_status pcsir_load(pcsir_ctx* ctx, const char* path) {
  if (!ctx || !path) return PCSIR_EINVAL;
  if (ctx->failed) return fail(ctx, PCSIR_ESTATE, "context failed earlier: " + ctx->err);
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, PCSIR_EINVAL, std::string("cannot open checkpoint ") + path);
  CkHead h;
  CkSur sr{};
  std::vector<float> params;
  uint64_t stored = 0;
  bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, CK_MAGIC, sizeof(CK_MAGIC)) == 0 &&
            h.version == CK_VERSION && (h.flags & ~1u) == 0u;
  if (ok && (h.flags & 1u)) {
    params.resize(PCSIR_SUR_NPARAMS);
    ok = std::fread(&sr, sizeof(sr), 1, f) == 1 &&
         std::fread(params.data(), sizeof(float), params.size(), f) == params.size();
  }
  ok = ok && std::fread(&stored, sizeof(stored), 1, f) == 1;
  char extra;
  ok = ok && std::fread(&extra, 1, 1, f) == 0;  // nothing may follow the hash
  std::fclose(f);
  if (!ok) return fail(ctx, PCSIR_EINVAL, std::string("not a pcSIR checkpoint of this version: ") + path);
  uint64_t hash = fnv1a(FNV_OFFSET, &h, sizeof(h));
  if (h.flags & 1u) {
    hash = fnv1a(hash, &sr, sizeof(sr));
    hash = fnv1a(hash, params.data(), params.size() * sizeof(float));
  }
  if (hash != stored) return fail(ctx, PCSIR_EINVAL, std::string("checkpoint is corrupt (hash): ") + path);
  if (!same_model(h.cfg, ctx->cfg))
    return fail(ctx, PCSIR_EINVAL, "checkpoint was written by a context with another model or state dtype");
  if (h.flags & 1u) {
    if (!ctx->sur_on)
      return fail(ctx, PCSIR_ESTATE, "the checkpoint holds a surrogate: attach one to the context before loading");
    pcsir_surrogate* sur = const_cast<pcsir_surrogate*>(ctx->sur.sur);
    double i0r = 0.0, sr_ = 0.0;
    sur_refs(sur, &i0r, &sr_);
    if (i0r != sr.i0_ref || sr_ != sr.sigma_ref)
      return fail(ctx, PCSIR_EINVAL, "the attached surrogate's i0_ref / sigma_ref differ from the checkpoint's");
    const pcsir_status st = pcsir_surrogate_set_params(sur, params.data(), sr.label_mean, sr.label_scale);
    if (st != PCSIR_OK) return fail(ctx, st, "setting the surrogate's parameters from the checkpoint");
    ctx->sur.frac = h.frac;
    ctx->sur.window = h.window;
    ctx->sur.max_err = h.max_err;
    ctx->sur.min_holdout = h.min_holdout;
  } else {
    ctx->sur_on = false;
  }
  ctx->sur_steps = h.salt;
  return PCSIR_OK;
}

pcsir_status pcsir_surrogate_last_check(pcsir_ctx* ctx, pcsir_surrogate_check* out) {
  if (!ctx || !out) return PCSIR_EINVAL;
  if (!ctx->sur_ran || ctx->last_kind != 1) return fail(ctx, PCSIR_ESTATE, "the last step did not use a surrogate");
  SurStats st{};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&st, ctx->sur.stats, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reading surrogate statistics");
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

pcsir_status pcsir_last_result(pcsir_ctx* ctx, pcsir_result* out) {
  if (!ctx || !out) return PCSIR_EINVAL;
  std::memcpy(out, ctx->host_res, sizeof(*out));
  return PCSIR_OK;
}

}  // extern "C"
