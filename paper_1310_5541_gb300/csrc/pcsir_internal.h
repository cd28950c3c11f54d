// Internal declarations shared by the host API and the kernel translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pcsir.h"
#include "../../include/pcsir_surrogate.h"

namespace pcsir {

// Per-step control block in device memory, zeroed at the start of every step.
struct Control {
  unsigned int nocc;          // occupied cells found so far (hash slots listed in occ[])
  unsigned int spare;
  unsigned int done_blocks;   // last-block-done counter of the weight reduction
  unsigned int err;           // PCSIR_DERR_* flags
  unsigned long long max_ll;  // ordered encoding of the maximum log-likelihood (bins)
  unsigned long long max_llq; // encoded maximum fixed-point log-likelihood (particles), 0 = none
  long long T_int;            // sum of the integer weights q_i (exact)
  double T_f;                 // sum of exp(ll_i - max)
  double T2_f;                // sum of exp(ll_i - max)^2
  double est[7];              // sum of exp(ll_i - max) * state_i (5 components in 2D, 7 in 3D)
  unsigned long long delta_hi, delta_lo;  // T_int / N as 64.64 fixed point
  unsigned long long u0_hi, u0_lo;        // u0 * T_int / N as 64.64 fixed point
  long long anchor[7];        // fixed-point anchors of the non-position components
  unsigned int tiles_done;    // finished tiles of the resampling kernel
  unsigned int tsum_done;     // finished tiles of the tile-sum kernel
  float inv_delta;            // 1 / Delta rounded to FP32 (first guesses of output indices)
  float spare_f;
};

// Limits of the fixed-point centre-of-mass sums.  Position offsets from the
// cell origin are < 8.5 * 2^31 (h <= 8) and other components are anchored at
// particle 0's value with |v - anchor| < 2^12; with N <= 2^26 no sum exceeds
// 2^62.
constexpr int64_t MAX_PARTICLES = int64_t(1) << 26;
constexpr double MAX_H = 8.0;

// Tile of the scan / resampling kernels.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

struct StepBuffers {
  // hash table over occupied cells (capacity hcap = 2^hbits >= 2 max_particles)
  unsigned long long* hkey;
  unsigned int* hcnt;
  long long* hsum;          // [5][hcap]
  unsigned int* hrank;      // hash slot -> bin index
  long long* hq;            // hash slot -> integer weight q
  double* hw;               // hash slot -> exp(ll - max)
  int hbits;
  // occupied bins, in discovery order (bin index)
  unsigned int* occ;        // bin -> hash slot
  int32_t* bin_xy;          // [2][max]
  uint32_t* bin_cnt;
  double* dummy;            // [5][max]
  double* bin_ll;
  // per particle
  void* prop;               // [5][max] state dtype
  unsigned int* pslot;      // particle -> hash slot
  double* ll;               // SIR per-particle log-likelihood (kept on request)
  long long* llq;           // SIR per-particle log-likelihood, fixed point 2^-32
  int32_t* anc;
  double* wout;
  long long* qout;          // integer weights of the resampling (kept on request)
  uint32_t* pbin;
  int64_t bin_stride;       // row stride of bin_xy / dummy (= max particles)
  // scan: per-tile sums of the integer weights and their exclusive prefixes
  long long* tile_sum;
  long long* tile_excl;
  // the tiles' outputs: tile t owns outputs [tile_lo[t], tile_lo[t + 1]); tile_ovx is the
  // exclusive prefix of the tiles' further output chunks past the first (max_tiles + 1 entries each)
  long long* tile_lo;
  int* tile_ovx;
  int64_t max_tiles;
  Control* ctl;
  pcsir_result* dres;
  int32_t* derr_out;        // where the last resampling tile publishes the step's device error flags
  int32_t* resampled_out;   // where it publishes whether the step resampled (nullptr: nowhere)
  // ESS-thresholded steps: with lw_out set the resampling kernel resamples only when
  // N_eff < ess_min and writes the carried fixed-point log-weights to lw_out
  long long* lw_out;
  double ess_min;
  int prop_bin_per_sm[2];   // resident blocks per SM of the propagate/bin kernel (small, large cell table)
  int big_table;            // 1: the propagate/bin kernel uses the large cell table
};

struct ModelParams {
  int P;
  int kind;
  double sigma;
  double bg;
  double sigma_xi;
  int coc;  // 1: dummies at cell centres (pcSIR-CoC)
};

// Optional stage events: when ev != nullptr the launchers record ev[1..] after
// their kernels (ev[0] is recorded by the caller before the first kernel).
struct StageEvents {
  cudaEvent_t* ev;  // 5 events of the current step, or nullptr
};

// Surrogate-assisted dummy likelihoods of one pcSIR step (pcsir_surrogate.cu):
// per-step counters and the held-out check's result, zeroed with the control
// block.
struct SurStats {
  unsigned int n_ho;       // held-out dummies found (entries past the list capacity are dropped)
  unsigned int n_clipped;  // dummies whose patch leaves the image
  unsigned int n_sig;      // significant held-out dummies
  unsigned int fallback;   // 1: every dummy takes the exact likelihood
  unsigned int bad;        // a prediction was not finite
  unsigned int n_nonfinite_err;
  double max_err;          // largest error over the significant held-out dummies
  double sum_sq;           // sum of squared errors over the held-out dummies
};

struct SurStep {
  const pcsir_surrogate* sur;
  unsigned long long salt;  // step counter since the attach
  double frac;              // held-out fraction
  int min_holdout;          // at least this many held-out dummies (when there are enough)
  int ho_cap;               // capacity of the held-out list
  double window;            // significance window below the maximum prediction
  double max_err;           // fallback threshold
  int* ho_bin;              // held-out list: bin index and exact log-likelihood
  double* ho_ll;
  SurStats* stats;
};

struct NoiseGen;  // counter-based process noise (pcsir_philox.cuh); ng != nullptr: noise ignored, FP32 only

// Kernel launchers (pcsir_kernels.cu / pcsir_resample.cu).
// sur == nullptr: exact likelihood of every dummy.  src_idx != nullptr: the input particle i is
// state[., src_idx[i]] (a resampling recorded as ancestors only, gathered here).
cudaError_t launch_pcsir_front(const StepBuffers& b, const ModelParams& m, int dtype, const void* state,
                               const void* noise, int64_t N, double h, const float* img, int W, int H,
                               int num_sms, cudaStream_t s, StageEvents se, const SurStep* sur = nullptr,
                               const int32_t* src_idx = nullptr, const NoiseGen* ng = nullptr);
// out[c * N + i] = src[c * N + idx[i]] for the 5 state components (idx == nullptr: a copy)
cudaError_t launch_gather_state(int dtype, const void* src, const int32_t* idx, void* out, int64_t N,
                                cudaStream_t s);
// largest image the surrogate's window-term buffer holds (pcsir_surrogate.cu)
int64_t sur_max_pixels(const pcsir_surrogate* s);
// 2 or 3: the surrogate's input geometry
int sur_dim(const pcsir_surrogate* s);
// surrogate predictions of the non-clipped dummies of a 3D step and the held-out check
cudaError_t launch_sur_step3(const SurStep& sp, const StepBuffers& b, double bg, double sigma_xy, const float* vol,
                             int W, int H, int D, cudaStream_t s);
// the surrogate's input normalisation constants (its creation config)
void sur_refs(const pcsir_surrogate* s, double* i0_ref, double* sigma_ref);
// surrogate predictions of the non-clipped dummies and the held-out check (pcsir_surrogate.cu)
cudaError_t launch_sur_step(const SurStep& sp, const StepBuffers& b, const ModelParams& m, const float* img, int W,
                            int H, cudaStream_t s);
// with_weights = 0: only the per-particle log-likelihoods and their maximum (the caller
// reduces the weights itself)
cudaError_t launch_sir_front(const StepBuffers& b, const ModelParams& m, int dtype, const void* state,
                             const void* noise, int64_t N, const float* img, int W, int H, int num_sms,
                             cudaStream_t s, StageEvents se, int keep, int with_weights = 1);
cudaError_t launch_logw_front(const StepBuffers& b, const double* logw, int64_t N, int num_sms,
                              cudaStream_t s);
// propagate + cells + centre-of-mass sums only (the first kernel of launch_pcsir_front)
cudaError_t launch_prop_bin(const StepBuffers& b, int dtype, const void* state, const void* noise, int64_t N,
                            double h, int num_sms, cudaStream_t s);
// weights, ESS and posterior mean from the per-particle fixed-point log-weights b.llq
// (kind 0: SIR result, 2: pcSIR result with per-particle weights)
cudaError_t launch_particle_weights(const StepBuffers& b, int dtype, int64_t N, int num_sms, int kind,
                                    cudaStream_t s);
// ESS-thresholded steps (pcsir_ess.cu): prior-weighted dummies, their likelihood and the
// carried log-weights (pcSIR), or the carried log-weights added to SIR's (lw_in: caller's array)
cudaError_t launch_pcsir_ess_front(const StepBuffers& b, const ModelParams& m, const long long* lw_in,
                                   const float* img, int W, int H, int64_t N, double h, int num_sms,
                                   cudaStream_t s);
cudaError_t launch_sir_ess_front(const StepBuffers& b, const long long* lw_in, int64_t N, int num_sms,
                                 cudaStream_t s);
cudaError_t prepare_kernels(int dtype, int prop_bin_per_sm[2]);
cudaError_t prepare_resample();
// integer-weight scale: q = rint(exp(ll - max) * 2^sq) with N * 2^sq <= 2^61
int weight_scale_bits(int64_t N);
cudaError_t launch_resample(const StepBuffers& b, int dtype, void* state_out, int64_t N, double u0,
                            int mode, int keep, int num_sms, cudaStream_t s);
// 3D state (7 components, FP32)
cudaError_t launch_resample7(const StepBuffers& b, float* state_out, int64_t N, double u0, int mode, int keep,
                             cudaStream_t s);
cudaError_t launch_resample_logw(const StepBuffers& b, const double* logw, int32_t* anc_out, int64_t N, double u0,
                                 cudaStream_t s);
cudaError_t launch_loglik(const ModelParams& m, const double* x, const double* y, const double* i0,
                          int64_t n, const float* img, int W, int H, double* out, int num_sms,
                          cudaStream_t s);

// resampling weight sources: per-cell integer weights (pcSIR), per-particle fixed-point
// log-likelihoods (SIR), caller log-weights, or per-particle integer weights already formed by
// the weight reduction into b.hq (ESS-thresholded steps; b.llq still holds the log-weights)
enum { WSRC_BINS = 0, WSRC_PARTICLES = 1, WSRC_LOGW = 2, WSRC_Q = 3 };

}  // namespace pcsir
