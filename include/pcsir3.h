/* pcSIR and SIR for 3D tracking: C ABI.
 *
 * The paper states Algorithms 1 and 2 for a general state and evaluates them
 * in 2D; its outlook names higher-dimensional settings.  This is the 3D form:
 *
 *   state (x, y, z, vx, vy, vz, I0), float32, structure-of-arrays [7][N] on the
 *   device, updated in place (resampled) by each step;
 *   nearly-constant-velocity dynamics with unit frame time (Section 5.1):
 *     x += vx + e_x, y += vy + e_y, z += vz + e_z, vx += e_vx, vy += e_vy,
 *     vz += e_vz, I0 += e_I, evaluated in float32 in this order;
 *   cells (Algorithm 2, Section 4.1): boxes of edges (hx, hy, hz) over
 *     position, b = floor((x + 1/2) / hx) per axis in float32, so unit edges
 *     are voxels centred on integers; |b| < 2^20 per axis (a particle beyond
 *     raises PCSIR_DERR_RANGE and is placed in cell (0, 0, 0));
 *   dummy: the centre of mass of the cell's members (all seven components);
 *   likelihood (Eq. object with an anisotropic Gaussian PSF, Eq. likelihood):
 *     the Poisson term z log(lambda / z) - (lambda - z) summed over a
 *     patch_xy x patch_xy x patch_z block of voxels centred on the nearest
 *     voxel (floor(x + 1/2), floor(y + 1/2), floor(z + 1/2)), with
 *     lambda = max(I0, 0) exp(-((u - x)^2 + (v - y)^2) / (2 s_xy^2)
 *                              - (w - z)^2 / (2 s_z^2)) + bg
 *     at voxel centres (u, v, w); voxels outside the volume contribute
 *     nothing.  The volume is float32 [D][H][W] on the device.
 *   resampling: systematic, every step, one uniform u0 (Algorithm 1/2), as
 *     in pcsir.h.
 *
 * Error behaviour, streams, graph capture and the result copy follow pcsir.h.
 */
#ifndef PCSIR3_H_
#define PCSIR3_H_

#include "pcsir.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcsir3_ctx pcsir3_ctx;

typedef struct pcsir3_config {
  int32_t patch_xy;       /* odd, 1 .. 63 */
  int32_t patch_z;        /* odd, 1 .. 63 */
  int32_t keep;           /* PCSIR_KEEP_* flags, as in pcsir.h */
  int32_t reserved;       /* must be 0 */
  double psf_sigma_xy;    /* > 0, voxels */
  double psf_sigma_z;     /* > 0, voxels */
  double bg;              /* > 0 */
  int64_t max_particles;  /* 1 .. 2^26 */
} pcsir3_config;

typedef struct pcsir3_result {
  double estimate[7];     /* posterior mean before resampling */
  double ess;
  double max_loglik;
  double sum_wtilde;
  int64_t n_particles;
  int64_t n_bins;         /* occupied cells (pcSIR), 0 for SIR */
  int32_t device_error;   /* PCSIR_DERR_* flags */
  int32_t kind;           /* 1 pcSIR, 0 SIR */
} pcsir3_result;

typedef struct pcsir3_outputs {
  int64_t n_particles;
  int64_t n_bins;
  int64_t bin_stride;        /* row stride of bin_xyz and dummy */
  const float* prop_state;   /* [7][N] propagated states */
  const int32_t* bin_xyz;    /* [3][bin_stride] cell indices */
  const uint32_t* bin_count; /* [n_bins] members per cell */
  const double* dummy;       /* [7][bin_stride] dummy states */
  const double* bin_loglik;  /* [n_bins] dummy log-likelihoods */
  const double* loglik;      /* [N] per-particle log-likelihoods (SIR, with PCSIR_KEEP_LOGLIK) */
  const uint32_t* particle_bin; /* [N] cell of each particle (with PCSIR_KEEP_PARTICLE_BIN) */
  const int32_t* ancestor;   /* [N] (with PCSIR_KEEP_ANCESTORS) */
  const double* weight;      /* [N] normalised weights (with PCSIR_KEEP_WEIGHTS) */
  const int64_t* qweight;    /* [N] integer weights of the resampling (with PCSIR_KEEP_QWEIGHTS) */
} pcsir3_outputs;

pcsir_status pcsir3_create(const pcsir3_config* cfg, pcsir3_ctx** out);
pcsir_status pcsir3_destroy(pcsir3_ctx* ctx);
const char* pcsir3_last_error(pcsir3_ctx* ctx);

/* One pcSIR step (Algorithm 2) in 3D on state [7][N] in place; noise [7][N]
   (device float32), u0 in [0, 1), cell edges hx, hy, hz in (0, 8].
   result_host (may be NULL) receives the step's scalars once the stream
   reaches the end of the step.  With a 3D surrogate attached
   (pcsir3_attach_surrogate), a volume of more voxels than the surrogate's
   max_pixels returns PCSIR_ERANGE before anything is launched. */
pcsir_status pcsir3_step(pcsir3_ctx* ctx, float* state, int64_t N, const float* volume, int32_t W, int32_t H,
                         int32_t D, double hx, double hy, double hz, const float* noise, double u0, void* stream,
                         pcsir3_result* result_host);

/* One SIR step (Algorithm 1) in 3D: the likelihood of every particle. */
pcsir_status sir3_step(pcsir3_ctx* ctx, float* state, int64_t N, const float* volume, int32_t W, int32_t H,
                       int32_t D, const float* noise, double u0, void* stream, pcsir3_result* result_host);

/* Intermediates of the last step (device pointers into the context, valid
   until its next step; reading n_bins synchronises the device). */
pcsir_status pcsir3_get_outputs(pcsir3_ctx* ctx, pcsir3_outputs* out);
/* The page-locked copy of the last step's result (synchronise the stream first). */
pcsir_status pcsir3_last_result(pcsir3_ctx* ctx, pcsir3_result* out);

/*
 * Batched multi-target 3D filtering: T independent targets, each its own
 * pcSIR filter (Algorithm 2) over the 3D state above, with its own particle
 * count, cell edges, PSF and patch, observed in one shared volume and
 * advanced together by one fixed sequence of kernels over all targets per
 * step (capturable as one CUDA graph).  The particles of all targets are
 * concatenated: target t owns particles [off_t, off_t + n_t) of the
 * [7][sum n_t] state, in target order.  The paper states its method for a
 * general state and names higher-dimensional settings as the extension; the
 * batching is a property of the library.
 */
typedef struct pcsir3_batch pcsir3_batch;

typedef struct pcsir3_target {
  int64_t n_particles;        /* >= 1 */
  double hx, hy, hz;          /* cell edges, (0, 8] voxels */
  double psf_sigma_xy;        /* > 0 */
  double psf_sigma_z;         /* > 0 */
  double bg;                  /* > 0 */
  int32_t patch_xy, patch_z;  /* odd, 1 .. 63 */
} pcsir3_target;

/* Device pointers to intermediates of the last batched step (valid until the
   next step).  Cells of all targets, n_bins of them in an unspecified order:
   bin_key = target << 54 | (bz + 2^17) << 36 | (by + 2^17) << 18 | (bx + 2^17),
   members, dummies ([7][bin_stride]) and dummy log-likelihoods. */
typedef struct pcsir3_batch_outputs {
  int64_t n_total;
  int64_t n_bins;
  int64_t bin_stride;
  const float* prop_state;      /* [7][n_total] propagated states */
  const uint64_t* bin_key;
  const uint32_t* bin_count;
  const double* dummy;
  const double* bin_loglik;
  const uint32_t* particle_slot;  /* [n_total] hash slot of each particle's cell (inspection) */
  const int32_t* ancestor;      /* [n_total] target-local ancestor of each output (PCSIR_KEEP_ANCESTORS) */
  const int64_t* qweight;       /* [n_total] integer weight of each particle (PCSIR_KEEP_QWEIGHTS) */
} pcsir3_batch_outputs;

/* Create the workspace for T targets (1 .. 1023, sum of n_particles <= 2^26);
   targets is a host array; keep: PCSIR_KEEP_ANCESTORS and/or
   PCSIR_KEEP_QWEIGHTS (per-particle outputs for inspection).  Cell indices
   must stay below 2^17 - 1 in magnitude (else PCSIR_DERR_RANGE).  Errors:
   PCSIR_EINVAL, PCSIR_ERANGE, PCSIR_ENOMEM, PCSIR_ECUDA. */
pcsir_status pcsir3_batch_create(const pcsir3_target* targets, int32_t T, int32_t keep, pcsir3_batch** out);
pcsir_status pcsir3_batch_destroy(pcsir3_batch* batch);
const char* pcsir3_batch_last_error(pcsir3_batch* batch);

/* One step of every target.  state: device float32 [7][sum n_t], read-write
   (resampled in place per target); volume: device float32 [D][H][W]; noise:
   device float32 [7][sum n_t]; u0: device float64 [T] systematic offsets in
   [0, 1).  Per target as pcsir3_step: propagate, cells of that target's
   edges, dummies, their likelihood (that target's PSF and patch), weights,
   systematic resampling within the target.  The per-target results are
   copied to page-locked memory of the batch at the end of the step.
   Allocates nothing; capturable in a CUDA graph. */
pcsir_status pcsir3_batched_step(pcsir3_batch* batch, float* state, const float* volume, int32_t W, int32_t H,
                                 int32_t D, const float* noise, const double* u0, void* stream);

/* Results of the last step, one per target (host array of T), and the step's
   PCSIR_DERR_* flags (device_error may be NULL).  Synchronises the device
   first, so the results are those of the last step enqueued. */
pcsir_status pcsir3_batch_results(pcsir3_batch* batch, pcsir3_result* out, int32_t T, int32_t* device_error);

/* Intermediates of the last step (synchronises the device).  Errors:
   PCSIR_EINVAL, PCSIR_ESTATE (no step yet), PCSIR_ECUDA. */
pcsir_status pcsir3_batch_get_outputs(pcsir3_batch* batch, pcsir3_batch_outputs* out);

#ifdef __cplusplus
}
#endif

#endif /* PCSIR3_H_ */
