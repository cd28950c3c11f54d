/*
 * pcsir.h - C ABI of the GB300 (sm_103a) piecewise-constant SIR particle filter.
 *
 * One call advances one particle filter by one time step k on the GPU, either
 * by plain sequential importance resampling (Algorithm 1 of Demirel et al.,
 * "Piecewise Constant Sequential Importance Sampling for Fast Particle
 * Filtering") or by its piecewise-constant variant pcSIR (Algorithm 2).
 *
 * Conventions shared by every entry point
 *  - All pointers named "device" point to memory of the current CUDA device;
 *    the library never frees caller memory.
 *  - State arrays are structure-of-arrays, component-major: element (d, i)
 *    of an N-particle state lives at state[d * N + i] with components
 *    d = 0..4 = (x, y, vx, vy, I0) (Section 5.1), in the context's state
 *    dtype (float or double).  Positions are in pixels; pixel (x, y) of an
 *    image is centred on integer coordinates (Eq. likelihood).
 *  - Images are float32, row-major: Z[y * W + x].
 *  - Work is enqueued on the given cudaStream_t (passed as void*, NULL = the
 *    legacy default stream) and is asynchronous: results are valid after the
 *    stream is synchronised.  Device memory is allocated only by the create
 *    calls (pcsir_create, pcsir3_create, pcsir_batch_create,
 *    pcsir_surrogate_create), by pcsir_batch_keep, and by the first
 *    pcsir_gemm_bf16 call of the process (a 4-byte error flag); no step call
 *    allocates, and every step call is capturable in a CUDA graph.
 *  - Every call returns a pcsir_status.  Argument errors are detected on the
 *    host before anything is enqueued.  Errors the GPU detects while running
 *    (non-finite or out-of-range states, a timed-out wait) are reported as
 *    bit flags in pcsir_result.device_error of that step.  Once a call has
 *    failed with PCSIR_ECUDA the context is unusable (sticky) and every later
 *    call returns PCSIR_ESTATE; pcsir_last_error() describes the failure.
 *  - A context is not thread-safe; steps on one context must be ordered on
 *    one stream (they share the context's workspace).
 */
#ifndef PCSIR_H_
#define PCSIR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcsir_ctx pcsir_ctx;

typedef enum pcsir_status {
  PCSIR_OK = 0,
  PCSIR_EINVAL = -1,    /* invalid argument (checked on the host) */
  PCSIR_ENOMEM = -2,    /* device allocation failed in pcsir_create */
  PCSIR_ECUDA = -3,     /* a CUDA call failed; the context becomes sticky-failed */
  PCSIR_ETIMEDOUT = -4, /* a bounded device wait gave up (pcsir_batch_results) */
  PCSIR_ESTATE = -5,    /* context already failed, or outputs requested before any step */
  PCSIR_ENOTSUP = -6,   /* combination of options not supported */
  PCSIR_ERANGE = -7     /* size beyond the limits fixed at pcsir_create */
} pcsir_status;

/* state dtype */
enum { PCSIR_F32 = 0, PCSIR_F64 = 1 };

/* likelihood of one image given a position (Eq. likelihood over the patch S_x) */
enum {
  /* Poisson log-likelihood ratio against a perfect fit, per pixel
     z*log(lambda/z) - (lambda - z) (0 when lambda = z, -lambda when z = 0) */
  PCSIR_LIK_POISSON = 0,
  /* the paper's Gaussian sum of squares, per pixel -(z - lambda)^2 / (2 sigma_xi^2) */
  PCSIR_LIK_SSE = 1
};

/* flags of pcsir_config.keep: optional per-particle outputs kept for inspection */
enum {
  PCSIR_KEEP_ANCESTORS = 1,    /* int32 ancestor index s(i) of every output particle */
  PCSIR_KEEP_WEIGHTS = 2,      /* float64 normalised weight w_k^i of every propagated particle */
  PCSIR_KEEP_PARTICLE_BIN = 4, /* uint32 bin index (into the bin arrays) of every particle */
  PCSIR_KEEP_LOGLIK = 8,       /* SIR: float64 log-likelihood of every propagated particle */
  PCSIR_KEEP_QWEIGHTS = 16     /* int64 integer weight q_i the resampling used for every particle */
};

/* bit flags of pcsir_result.device_error */
enum {
  PCSIR_DERR_RANGE = 1,     /* non-finite state, |position| >= 2^30, cell index or spread beyond limits */
  PCSIR_DERR_TIMEOUT = 2,   /* a bounded inter-block wait gave up (results of the step are invalid) */
  PCSIR_DERR_NONFINITE = 4, /* a log-likelihood was not finite (its weight was set to 0) */
  PCSIR_DERR_ZEROSUM = 8    /* every weight was zero: no resampling possible (state left propagated) */
};

/*
 * Model and limits, fixed for the life of a context.
 * psf_sigma, bg: Gaussian point-spread function of Eq. (object),
 *   lambda(px, py) = max(I0, 0) * exp(-((px - x)^2 + (py - y)^2) / (2 psf_sigma^2)) + bg,
 *   point-sampled at pixel centres.
 * patch: odd side P of the square patch S_x of Eq. (likelihood), centred on the
 *   pixel nearest the evaluated position, (floor(x + 0.5), floor(y + 0.5));
 *   pixels outside the image contribute nothing.
 * max_particles: largest N any step of this context will use (1 .. 2^26).
 */
typedef struct pcsir_config {
  int32_t state_dtype;   /* PCSIR_F32 or PCSIR_F64 */
  int32_t lik_kind;      /* PCSIR_LIK_POISSON or PCSIR_LIK_SSE */
  int32_t patch;         /* odd, 1 .. 127 */
  int32_t keep;          /* PCSIR_KEEP_* flags */
  double psf_sigma;      /* > 0, pixels */
  double bg;             /* background intensity; > 0 for PCSIR_LIK_POISSON */
  double sigma_xi;       /* > 0; used by PCSIR_LIK_SSE only */
  int64_t max_particles; /* 1 .. 2^26 */
  int32_t dummy;         /* PCSIR_DUMMY_COM (0) or PCSIR_DUMMY_COC (1), see below */
  int32_t reserved;      /* must be 0 */
} pcsir_config;

/* Placement of the dummy particle of a cell (Section 5.4): at the centre of
   mass of its members (pcSIR-CoM, Algorithm 2), or at the cell's geometric
   centre ((bx + 1/2) h - 1/2, (by + 1/2) h - 1/2) for the binned position
   with the members' mean for the other components (pcSIR-CoC). */
#define PCSIR_DUMMY_COM 0
#define PCSIR_DUMMY_COC 1

/* Scalars of one step, in host memory (see result_host below). */
typedef struct pcsir_result {
  double estimate[5];   /* posterior mean of (x, y, vx, vy, I0) before resampling */
  double ess;           /* effective sample size 1 / sum_i w_i^2 (Algorithm 1) */
  double max_loglik;    /* max over particles of the log-likelihood */
  double sum_wtilde;    /* sum_i exp(ll_i - max_loglik); w_i = exp(ll_i - max_loglik) / sum_wtilde */
  int64_t n_particles;  /* N of the step */
  int64_t n_bins;       /* pcSIR: occupied bins B; SIR: 0 */
  int32_t device_error; /* PCSIR_DERR_* flags, 0 if none */
  int32_t kind;         /* 0 = SIR step, 1 = pcSIR step */
  int32_t resampled;    /* 1 if the step resampled (always, except in the ESS-thresholded steps) */
  int32_t reserved;
} pcsir_result;

/* Device pointers to intermediates of the most recent step of a context,
   valid until the next step on that context (read them after synchronising).
   Bin arrays hold the B occupied bins in an unspecified order that is the
   same across all bin arrays; NULL where the step kind or keep flags do not
   produce the array. */
typedef struct pcsir_outputs {
  int64_t n_particles;
  int64_t n_bins;
  int64_t bin_stride;            /* element (d, b) of bin_xy / dummy is at [d * bin_stride + b] */
  const void* prop_state;        /* [5][N] propagated states x~_k (state dtype) */
  const int32_t* bin_xy;         /* [2][bin_stride] cell indices (bx, by), bx = floor((x + 0.5) / h) */
  const uint32_t* bin_count;     /* [B] members per bin */
  const double* dummy;           /* [5][bin_stride] dummy states (mean state of each bin) */
  const double* bin_loglik;      /* [B] log-likelihood of each dummy */
  const double* loglik;          /* SIR: [N] log-likelihood of each propagated particle (PCSIR_KEEP_LOGLIK) */
  const uint32_t* particle_bin;  /* [N] bin index of each particle (PCSIR_KEEP_PARTICLE_BIN) */
  const int32_t* ancestor;       /* [N] s(i) for each output particle i (PCSIR_KEEP_ANCESTORS) */
  const double* weight;          /* [N] normalised weights (PCSIR_KEEP_WEIGHTS) */
  /* [N] integer weights (PCSIR_KEEP_QWEIGHTS): q_i = rint(w~_i 2^s), w~_i = exp(log w_i - max),
     with N 2^s <= 2^61 so every cumulative sum C_j = q_0 + ... + q_j is exact.  The resampling
     of the step is exactly systematic over them: output i takes the first j with
     C_j > (i + u0) C_{N-1} / N (up to a 2^-64 relative rounding of that bound). */
  const int64_t* qweight;
} pcsir_outputs;

/* Create a context on the current CUDA device: validates cfg and allocates
   all workspace for up to cfg->max_particles particles.  On success *out
   receives the context; on failure *out is set to NULL.
   Errors: PCSIR_EINVAL (bad cfg or NULL out), PCSIR_ENOMEM, PCSIR_ECUDA. */
pcsir_status pcsir_create(const pcsir_config* cfg, pcsir_ctx** out);

/* Release a context and its workspace (synchronises the device first).
   NULL is accepted and ignored. */
pcsir_status pcsir_destroy(pcsir_ctx* ctx);

/*
 * One pcSIR step (Algorithm 2, resampling every step).
 *   state  device [5][N], state dtype, read-write: on entry the states
 *          x_{k-1} (all weights equal, as after resampling), on return the
 *          resampled states x_k.
 *   N      particles, 1 .. max_particles.
 *   image  device float32 [H][W], the observation z_k, read-only.
 *   h      cell edge in pixels, 0 < h <= 8.  Cells are [b h - 0.5, (b+1) h - 0.5)
 *          on each axis, so h = 1 cells are the image pixels (pcSIR-1x1) and
 *          h = 0.5 quarters them (pcSIR-2x2) (Section 4.2).
 *   noise  device [5][N] in the state dtype: the process noise e added by the
 *          nearly-constant-velocity transition (Section 5.1),
 *          x += vx + e_x, y += vy + e_y, vx += e_vx, vy += e_vy, I0 += e_I0.
 *   u0     systematic-resampling offset in [0, 1): output particle i takes
 *          the first particle l whose inclusive cumulative weight exceeds
 *          (i + u0) / N of the total.
 *   stream cudaStream_t (as void*).
 *   result_host  NULL, or host memory (page-locked for a truly asynchronous
 *          copy) that receives the step's pcsir_result once the stream has
 *          reached the end of the step.
 * Steps: propagate, cell index, per-cell centre of mass (the dummy),
 * likelihood of the dummies only, the dummy's weight copied to its members,
 * normalisation, ESS, posterior mean, systematic resampling.
 * Errors: PCSIR_EINVAL (NULL pointers, N or h out of range, W or H < 1,
 * u0 outside [0,1)), PCSIR_ERANGE (N > max_particles), PCSIR_ECUDA,
 * PCSIR_ESTATE.
 */
pcsir_status pcsir_step(pcsir_ctx* ctx, void* state, int64_t N, const float* image,
                        int32_t W, int32_t H, double h, const void* noise, double u0,
                        void* stream, pcsir_result* result_host);

/*
 * pcsir_step with the process noise drawn in the propagation kernel instead
 * of read from a device array: the nearly-constant-velocity increments of
 * Section 5.1, e_d = q_d z_d for the five components, with z standard
 * normals from the counter-based generator Philox4x32-10 (Salmon, Moraes,
 * Dror and Shaw, SC 2011) and the Box-Muller transform.
 *   q      host double[5]: standard deviations of the increments of x, y,
 *          vx, vy, I0 (finite, >= 0), rounded to float.
 *   seed   64-bit key of the generator.
 *   frame  0 .. 2^32 - 1: particle i of frame k draws from the counters
 *          (i mod 2^32, i div 2^32, k, 0) and (..., 1); the same (seed, frame)
 *          gives the same noise, whatever N or the launch shape.
 * The transform uses only correctly rounded single-precision operations and
 * series for its logarithm, sine and cosine, so that a CPU implementation of
 * the same steps reproduces the noise bit for bit; the normals agree with the
 * exact transform to a few units in the last place.  Per FP32 particle the
 * propagation reads 24 bytes instead of 44 (no noise array): the end-to-end
 * path then copies only the image per step.  FP32 state only
 * (PCSIR_ENOTSUP otherwise); PCSIR_EINVAL for a NULL or invalid q or a frame
 * of 2^32 or more.  Other arguments, outputs and errors as pcsir_step.
 */
pcsir_status pcsir_step_philox(pcsir_ctx* ctx, void* state, int64_t N, const float* image, int32_t W, int32_t H,
                               double h, const double* q, uint64_t seed, uint64_t frame, double u0, void* stream,
                               pcsir_result* result_host);

/*
 * Deferred resampling: a run of pcSIR steps (Algorithm 2, resampling every
 * step) whose particle set lives in the context between steps.  pcsir_step
 * gathers the resampled states x_k^i = x~_k^{a(i)} into the caller's buffer
 * (read and write 5 states per particle) only for the next step to read them
 * back; here the resampling records the ancestors a(i) and the next step's
 * propagation reads x~_k^{a(i)} itself.  Same filter, same numbers: each
 * step's propagated states, cells, dummies, likelihoods, weights, results and
 * ancestors equal pcsir_step's bit for bit on the same inputs; the saving is
 * the gather (40 B per FP32 particle and step).
 *
 * pcsir_deferred_begin copies `state` ([5][N], the states x_0, all weights
 *   equal) into the context on `stream` and starts a run of N particles.  On
 *   its first call it allocates the run's second state buffer and ancestor
 *   array (24 B per FP32 particle, 44 B FP64); PCSIR_ENOMEM if that fails.
 * pcsir_deferred_step: one step of the run, arguments as pcsir_step.  The
 *   outputs (pcsir_get_outputs) are those of pcsir_step; `ancestor` is always
 *   filled (it is the run's ancestor array).
 * pcsir_deferred_state writes the run's current resampled states x_k into
 *   `state` ([5][N], caller-owned, device) on `stream`; the run continues.
 * Any other step on the context (pcsir_step, sir_step, the ESS steps) ends
 * the run; pcsir_deferred_step then returns PCSIR_ESTATE until the next
 * begin.  Not with an attached surrogate (PCSIR_ENOTSUP).  Checkpoints
 * (pcsir_save) do not hold the run's states: write them out with
 * pcsir_deferred_state.  Errors otherwise as pcsir_step.
 */
pcsir_status pcsir_deferred_begin(pcsir_ctx* ctx, const void* state, int64_t N, void* stream);
pcsir_status pcsir_deferred_step(pcsir_ctx* ctx, const float* image, int32_t W, int32_t H, double h,
                                 const void* noise, double u0, void* stream, pcsir_result* result_host);
pcsir_status pcsir_deferred_state(pcsir_ctx* ctx, void* state, void* stream);
/* A step of the run with the noise drawn in the kernel, as pcsir_step_philox. */
pcsir_status pcsir_deferred_step_philox(pcsir_ctx* ctx, const float* image, int32_t W, int32_t H, double h,
                                        const double* q, uint64_t seed, uint64_t frame, double u0, void* stream,
                                        pcsir_result* result_host);

/* One SIR step (Algorithm 1, bootstrap proposal, resampling every step): as
   pcsir_step without the bins; the likelihood is evaluated for every particle. */
pcsir_status sir_step(pcsir_ctx* ctx, void* state, int64_t N, const float* image,
                      int32_t W, int32_t H, const void* noise, double u0,
                      void* stream, pcsir_result* result_host);

/* ESS-thresholded steps: Algorithms 1 and 2 with their test on the effective
 * sample size (Section 3, Algorithm 1: resample when N_eff < N_thr), the
 * weights being carried to the next step when the test fails.  pcsir_step / sir_step are the case that always
 * resamples.
 *
 * logw: device int64 [N], read and written, the particles' carried
 *   log-weights in fixed point: log w = logw * 2^-32.  On entry, what the
 *   previous call returned (all zeros for uniform weights, e.g. on the first
 *   step): values <= 0 whose maximum is 0, or INT64_MIN for a particle of
 *   zero weight.  On return: all zeros if the step resampled, else the step's
 *   log-weights log w_{k-1} + log p(z | x_k) minus their maximum.
 * ess_min: the step resamples when N_eff < ess_min (ess_min > N: every step;
 *   ess_min <= 0: never).  N_eff = (sum w)^2 / sum w^2 is result->ess.
 * pcsir_step_ess: each cell's dummy is the mean of its members weighted by
 *   w_{k-1} (Section 4: a centre of mass that weighs each member by its weight); the
 *   members' weights are multiplied by the dummy's likelihood.  The weighted
 *   sums are formed in FP32 per block and FP64 across blocks (within a few
 *   FP32 units in the last place of the weighted offsets, and not bit-for-bit
 *   reproducible).  Each member's weight is taken relative to the largest
 *   carried weight in its own cell, so a cell keeps its weighted mean however
 *   far below the other cells it lies; a member below about e^-87 of its
 *   cell's largest adds nothing (FP32 exponential), and a cell none of whose
 *   members carries weight (all INT64_MIN) takes the plain mean.
 * Without resampling the state becomes the propagated state and
 * PCSIR_KEEP_ANCESTORS gives the identity; result->resampled tells which branch
 * the step took.  FP32 state only (PCSIR_ENOTSUP for FP64), and not with an
 * attached surrogate (PCSIR_ENOTSUP).  Other arguments, errors, streams and
 * graph capture as pcsir_step / sir_step.
 */
pcsir_status pcsir_step_ess(pcsir_ctx* ctx, void* state, int64_t* logw, int64_t N, const float* image,
                            int32_t W, int32_t H, double h, const void* noise, double u0, double ess_min,
                            void* stream, pcsir_result* result_host);
pcsir_status sir_step_ess(pcsir_ctx* ctx, void* state, int64_t* logw, int64_t N, const float* image,
                          int32_t W, int32_t H, const void* noise, double u0, double ess_min,
                          void* stream, pcsir_result* result_host);

/* Log-likelihood (Eq. likelihood with the context's model) of n positions:
   x, y, I0 device float64 [n], out device float64 [n].  The same device code
   the steps use; exposed for tests and for labelling likelihood data. */
pcsir_status pcsir_loglik(pcsir_ctx* ctx, const double* x, const double* y, const double* I0,
                          int64_t n, const float* image, int32_t W, int32_t H, double* out,
                          void* stream);

/* Systematic resampling alone (Algorithm 1 resampling step): ancestors of N
   outputs from N log-weights.  logw device float64 [N] (weights are
   exp(logw - max logw)); ancestors device int32 [N].  Uses the step's scan
   and resampling kernels; N <= max_particles. */
pcsir_status pcsir_resample(pcsir_ctx* ctx, const double* logw, int64_t N, double u0,
                            int32_t* ancestors, void* stream);

/* Per-stage timing.  pcsir_timing_enable(ctx, max_steps) creates CUDA events
   for max_steps steps (max_steps = 0 disables timing and frees them); every
   later step records an event before its first kernel and after each of its
   four kernel stages, into slot (step count mod max_steps), without any
   synchronisation.  pcsir_timing_read(ctx, ms, capacity, &n_steps) waits for
   the recorded steps (since enable or the previous read, at most max_steps)
   and writes, for step s, the durations in milliseconds of stage j = 0..3 to
   ms[4 s + j]: pcSIR = (propagate + cells + centre-of-mass sums, dummies +
   likelihood, weight reduction, scan + resample), SIR = (propagate +
   likelihood, weight reduction, 0, scan + resample).  capacity is the length
   of ms in floats.  Errors: PCSIR_EINVAL, PCSIR_ESTATE (timing not enabled),
   PCSIR_ECUDA. */
pcsir_status pcsir_timing_enable(pcsir_ctx* ctx, int32_t max_steps);
pcsir_status pcsir_timing_read(pcsir_ctx* ctx, float* ms, int32_t capacity, int32_t* n_steps);

/* Systematic resampling for callers that cannot allocate device memory (the
   paper has no counterpart: this is a property of the library, not of the
   method).  Some callers may not call cudaMalloc: a host application whose
   device-memory budget is fixed and handed out at start-up, a framework
   whose caching allocator already owns the free memory, or a real-time loop
   that must not take the device-wide synchronisation an allocation can
   cause.  This entry point needs no context and allocates nothing: its
   scratch is a fixed array of about 17 KB in the library's own device
   memory, held by every GPU that loads the library until the process exits.
     logw       device float64 [N] log-weights (weights exp(logw - max logw)).
     N          1 .. 2^22 (4,194,304); larger N returns PCSIR_ERANGE.
     u0         systematic offset in [0, 1).
     ancestors  device int32 [N], receives s(i) for every output i; the same
                values pcsir_resample returns for the same inputs.
   If no weight is positive (every log-weight -inf or NaN) there is no
   distribution to sample: the call still returns PCSIR_OK, with the identity
   ancestors s(i) = i, as pcsir_resample does; a caller that may pass such
   weights checks them itself.
   The first call on each device (with that device current) makes the
   device's primary context current, looks up the scratch array's address and
   sets a kernel attribute; make that first call before any stream capture.
   The lookup is cached per device and CUDA context: after a device reset the
   next call repeats it (again outside any capture).  All calls on a device
   share the one scratch array: calls whose work may overlap on the GPU
   (different streams without ordering) race on it and must not be issued.
   logw, ancestors and the stream must belong to the current device.
   Errors: PCSIR_EINVAL, PCSIR_ERANGE, PCSIR_ECUDA. */
pcsir_status pcsir_resample_noalloc(const double* logw, int64_t N, double u0, int32_t* ancestors, void* stream);

/* Intermediates of the last step (see pcsir_outputs).  Host call, no sync. */
pcsir_status pcsir_get_outputs(pcsir_ctx* ctx, pcsir_outputs* out);

/* Copy of the last step's pcsir_result kept by the context in page-locked
   memory (valid after the stream of that step is synchronised). */
pcsir_status pcsir_last_result(pcsir_ctx* ctx, pcsir_result* out);

/* Checkpoint and resume (the paper has no counterpart: a property of the
 * library).  Between steps a context carries, besides workspace, only the
 * state of an attached likelihood surrogate (pcsir_surrogate.h): its network
 * parameters and label normalisation, its held-out settings, and the count of
 * surrogate-assisted steps since the attach, which salts the held-out
 * selection of the next step.  The filter's own state (particle states,
 * carried log-weights, frame index, seeds) is the caller's and is saved by
 * the caller.
 *
 * pcsir_save(ctx, path) writes that context state to the file path (through
 * path.tmp, renamed on success).  pcsir_load(ctx, path) restores it into ctx,
 * which must have been created with the same model and state dtype (every
 * pcsir_config field but keep; else PCSIR_EINVAL).  When the checkpoint holds
 * a surrogate, attach one (created with the same i0_ref and sigma_ref) to ctx
 * first: pcsir_load writes the saved parameters into it (its Adam moments are
 * zeroed) and restores the held-out settings and the step count, so that the
 * steps after a load repeat, bit for bit, those that followed the save.
 * Without a surrogate record pcsir_load detaches any attached surrogate.
 * Both calls synchronise the device and may not be captured in a CUDA graph.
 * File layout: an 8-byte magic "PCSIRCK1", version 1, flags, the pcsir_config,
 * the held-out state, the surrogate record, and an FNV-1a hash of all of it,
 * in host byte order.  Errors: PCSIR_EINVAL (NULL arguments, unreadable,
 * unwritable, corrupt or foreign file, model mismatch), PCSIR_ESTATE (context
 * failed, or a surrogate record without an attached surrogate), PCSIR_ECUDA. */
pcsir_status pcsir_save(pcsir_ctx* ctx, const char* path);
pcsir_status pcsir_load(pcsir_ctx* ctx, const char* path);

/* Human-readable description of the last error on ctx (never NULL). */
const char* pcsir_last_error(pcsir_ctx* ctx);

/*
 * Batched multi-target filtering: T independent targets, each its own pcSIR
 * filter (Algorithm 2) with its own particle count, PSF, patch and cell edge,
 * observed in one shared image and advanced together by one persistent
 * cooperative kernel launch per step.  FP32 state, Poisson likelihood.
 * The particles of all targets are concatenated: target t owns particles
 * [off_t, off_t + n_t) of the [5][sum n_t] state, in target order.
 */
typedef struct pcsir_batch pcsir_batch;

typedef struct pcsir_target {
  int64_t n_particles;  /* >= 1 */
  double h;             /* cell edge, 0 < h <= 8 */
  double psf_sigma;     /* > 0 */
  double bg;            /* > 0 */
  int32_t patch;        /* odd, 1 .. 63 */
  int32_t pad;
} pcsir_target;

/* Create the workspace for T targets (1 .. 2047, sum of n_particles <= 2^26);
   targets is a host array.  Errors: PCSIR_EINVAL, PCSIR_ERANGE, PCSIR_ENOMEM,
   PCSIR_ENOTSUP (no cooperative launch), PCSIR_ECUDA. */
pcsir_status pcsir_batch_create(const pcsir_target* targets, int32_t T, pcsir_batch** out);
pcsir_status pcsir_batch_destroy(pcsir_batch* batch);

/* Blocks per SM of the persistent kernel (default: the most that fit, 2).
   A launch-shape knob for the autotuner; results do not depend on it.
   Errors: PCSIR_EINVAL, PCSIR_ERANGE (more than fit), PCSIR_ECUDA. */
pcsir_status pcsir_batch_set_grid(pcsir_batch* batch, int32_t blocks_per_sm);

/* Size of the persistent kernel's block-private cell table: 2^table_bits
   slots, table_bits in 9 .. 11 (default 10), a launch-shape knob for the
   autotuner (results do not depend on it).  A larger table holds more cells
   before a block spills to the global table but takes more shared memory
   (2^11: one block per SM); the grid shrinks to what fits.  Errors:
   PCSIR_EINVAL, PCSIR_ERANGE, PCSIR_ECUDA. */
pcsir_status pcsir_batch_set_table(pcsir_batch* batch, int32_t table_bits);

/* One step of every target.  state: device float32 [5][sum n_t], read-write
   (resampled in place per target); image: device float32 [H][W]; noise:
   device float32 [5][sum n_t] process noise (Section 5.1); u0: device float64
   [T] systematic offsets in [0, 1).  Each target's particles are propagated,
   binned (cells of that target's h), reduced to dummies, weighted by the
   dummies' likelihood (that target's PSF and patch) and resampled within the
   target, as pcsir_step does for one target.  The per-target pcsir_result
   array is copied to page-locked memory owned by the batch; read it with
   pcsir_batch_results after synchronising.  Capturable in a CUDA graph. */
pcsir_status pcsir_batched_step(pcsir_batch* batch, float* state, const float* image, int32_t W, int32_t H,
                                const float* noise, const double* u0, void* stream);

/* Deferred resampling of a batch (the paper has no counterpart; the same
   filter as pcsir_batched_step, with the resampled states never written out
   between steps).  pcsir_batch_deferred_begin copies `state` (device float32
   [5][sum n_t], the states x_0 of every target, all weights equal) into the
   batch on `stream` and starts a run; on its first call it allocates a second
   propagated-state buffer and an ancestor array (24 B per particle), else
   PCSIR_ENOMEM.  pcsir_batched_deferred_step is one step of every target,
   image, noise and u0 as pcsir_batched_step: the resampling phase records
   each output particle's ancestor instead of moving the states, and the next
   step's propagation reads its input states through those ancestors (24 B
   per particle instead of the resampling's 40 B of states).  Results,
   outputs, bins and kept arrays are those of pcsir_batched_step.
   pcsir_batch_deferred_state writes the run's current resampled states into
   `state` ([5][sum n_t], caller-owned, device) on `stream`; the run
   continues.  A pcsir_batched_step ends the run: the deferred calls then
   return PCSIR_ESTATE until the next begin.  A captured graph of deferred
   steps alternates the two state buffers step by step: replay it with an even
   number of steps per graph.  Errors otherwise as pcsir_batched_step. */
pcsir_status pcsir_batch_deferred_begin(pcsir_batch* batch, const float* state, void* stream);
pcsir_status pcsir_batched_deferred_step(pcsir_batch* batch, const float* image, int32_t W, int32_t H,
                                         const float* noise, const double* u0, void* stream);
pcsir_status pcsir_batch_deferred_state(pcsir_batch* batch, float* state, void* stream);

/* Results of the last step, one per target (out: host array of T), and the
   step's PCSIR_DERR_* flags (device_error may be NULL).  Synchronises the
   device first, so the results are those of the last step enqueued.  Returns PCSIR_ETIMEDOUT (with out and
   *device_error filled) when the flags hold PCSIR_DERR_TIMEOUT: a grid-barrier
   wait of the step gave up, every block left the kernel, and the step's
   results are invalid.  The batch stays usable: the next step first clears
   the cell table the interrupted step may have left partly filled. */
pcsir_status pcsir_batch_results(pcsir_batch* batch, pcsir_result* out, int32_t T, int32_t* device_error);

/* Device pointers of the last step's propagated states (5 rows of sum n_t
   values, row r at prop_state + r * row_stride; row_stride is sum n_t rounded
   up to a multiple of 4 so that every row starts on a 16-byte boundary) and
   per-particle cell slots (for inspection), and the total particle count.
   Any out-pointer may be NULL. */
pcsir_status pcsir_batch_outputs(pcsir_batch* batch, const float** prop_state, int64_t* row_stride,
                                 const unsigned int** particle_slot, int64_t* n_total);

/* Device pointers to the last step's occupied cells of all targets (n_bins of
   them, in an unspecified order): keys (target << 52 | (by + 2^25) << 26 |
   (bx + 2^25)), member counts and dummy log-likelihoods.  Reading n_bins
   synchronises the device. */
pcsir_status pcsir_batch_bins(pcsir_batch* batch, const uint64_t** keys, const uint32_t** counts,
                              const double** loglik, int64_t* n_bins);

const char* pcsir_batch_last_error(pcsir_batch* batch);

/* Bounded waits of the persistent kernel (failure detection; the paper has no
   counterpart).  Each grid-barrier wait polls at most max_polls times (default
   4,194,304, with a 64 ns sleep per poll) before it gives up with
   PCSIR_DERR_TIMEOUT.  unreachable_barrier in 0 .. 6 makes that barrier of the
   step wait for one block more than the grid holds, a release that never
   comes, so that its wait runs out: a test of the timeout path that needs no
   fault.  -1 (the default) makes every barrier reachable.  Applies to steps
   launched (or graphs captured) after the call.  Errors: PCSIR_EINVAL. */
pcsir_status pcsir_batch_set_wait(pcsir_batch* batch, int32_t max_polls, int32_t unreachable_barrier);

/* Per-particle outputs of later steps, kept for inspection: keep is a
   combination of PCSIR_KEEP_ANCESTORS (int32 [sum n_t]: for output particle i
   of target t, at off_t + i, the index within the target of its ancestor) and
   PCSIR_KEEP_QWEIGHTS (int64 [sum n_t]: the integer weight q of each
   propagated particle, q = rint(exp(ll - max_t) 2^s_t) with n_t 2^s_t <= 2^61;
   each target is resampled exactly systematically over its own q).  Allocates
   the arrays (once); call it before capturing steps in a graph.
   pcsir_batch_kept returns the device pointers (NULL where not kept), valid
   for the life of the batch; read them after the step's stream is
   synchronised.  Errors: PCSIR_EINVAL, PCSIR_ENOMEM, PCSIR_ESTATE. */
pcsir_status pcsir_batch_keep(pcsir_batch* batch, int32_t keep);
pcsir_status pcsir_batch_kept(pcsir_batch* batch, const int32_t** ancestor, const int64_t** qweight);

/* Durations in ms of the last batched step's seven phases (set-up, propagate
   and cells, dummies and likelihood, weights, tile sums, per-target scan,
   resampling), from global-timer readings of block 0 at each grid barrier;
   ms holds n >= 7 values.  Synchronises the device.  Diagnostics only: the
   paper has no counterpart. */
pcsir_status pcsir_batch_phase_times(pcsir_batch* batch, double* ms, int32_t n);

/* BF16 tensor-core GEMM (tcgen05, FP32 accumulation), the building block of
   the likelihood surrogate (the paper has no counterpart; exposed for tests).
   C[m * ldc + n] (+)= sum_k A[m * sam + k * sak] * B[n * sbn + k * sbk] for
   m < M, n < N, k < K; A and B device bf16 (as uint16_t), C device float32.
   accumulate != 0 adds to C.  The first call of the process allocates a
   4-byte device error flag (kept until exit).  Errors: PCSIR_EINVAL,
   PCSIR_ENOMEM, PCSIR_ECUDA. */
pcsir_status pcsir_gemm_bf16(const uint16_t* A, int64_t sam, int64_t sak, const uint16_t* B, int64_t sbn,
                             int64_t sbk, float* C, int64_t ldc, int32_t M, int32_t N, int32_t K, int32_t accumulate,
                             void* stream);

/* Library version string. */
const char* pcsir_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PCSIR_H_ */
