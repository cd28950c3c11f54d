/* Learned likelihood surrogate for the pcSIR step: C ABI.
 *
 * The paper has no counterpart: this is an addition that leaves the method
 * unchanged.  In Algorithm 2 the dummy particle of each occupied cell is
 * weighted by the likelihood of Eq. likelihood (Gaussian PSF of Eq. object
 * rendered over a P x P patch); the surrogate predicts that log-likelihood
 * with a small network evaluated on the tensor cores, and the exact
 * likelihood stays both its fallback and the measure of its error on a
 * held-out set of dummies at every step.
 *
 * Network (all sizes fixed): 445 inputs -> 256 -> 256 -> 1 with SiLU
 * activations, silu(t) = t / (1 + exp(-t)).  Inputs of a state (x, y, I0)
 * against an image (row-major H x W float32, pixel (c, r) centred at
 * (c, r)):
 *   0..440   the 21 x 21 patch centred on the nearest pixel
 *            (cx, cy) = (floor(x + 0.5), floor(y + 0.5)), row by row from
 *            (cx - 10, cy - 10), as (z - bg) / i0_ref;
 *   441, 442 2 (x - cx), 2 (y - cy);
 *   443, 444 I0 / i0_ref, sigma / sigma_ref (sigma = the PSF width).
 * A state whose patch leaves the image ("clipped") is never given to the
 * network.
 *
 * What the network predicts.  With lambda = bg + I0 g (g the PSF) the
 * Poisson term of the likelihood splits, pixel by pixel, into a part that
 * depends on the image alone and a part that involves the spot:
 *   z log(lambda / z) - (lambda - z)
 *     = [z - z log z + z log bg - bg] + [z log(1 + I0 g / bg) - I0 g].
 * The first part summed over the window, T(cx, cy) = sum (z - z log z) +
 * log(bg) sum z - 441 bg (0 log 0 = 0), is computed for every window of a
 * frame by a box filter (per-pixel terms in FP32, sums in double-float,
 * result rounded to FP32).  The
 * network learns the residual r = ll - T from the training labels; the
 * predicted log-likelihood is T + label_mean + label_scale * out, where out
 * is the network output.  Weights W1 (256 x 445) and W2 (256 x 256) enter the
 * tensor cores as bf16 copies of FP32 master weights; activations are bf16,
 * accumulation FP32; biases, the output layer and the head run in FP32.
 *
 * Packed parameter layout (float32, PCSIR_SUR_NPARAMS values, in order):
 * W1 [256][445] row-major, b1 [256], W2 [256][256] row-major, b2 [256],
 * w3 [256], b3 [1].
 *
 * 3D surrogate (geometry 3; the 3D step of pcsir3.h, whose likelihood is the
 * Poisson term over an 11 x 11 x 7 voxel patch): 852 inputs -> 256 -> 256 -> 1,
 *   0..846   the 11 x 11 x 7 patch centred on the nearest voxel (cx, cy, cz),
 *            x fastest, then y, then z, from (cx - 5, cy - 5, cz - 3), as
 *            (z - bg) / i0_ref;
 *   847..849 2 (x - cx), 2 (y - cy), 2 (z - cz);
 *   850, 851 I0 / i0_ref, sigma_xy / sigma_ref.
 * The window term sums the image-only part over the 847 voxels of the window
 * (separable passes along x, y and z, sums in double-float); the packed
 * parameters (PCSIR_SUR3_NPARAMS) are W1 [256][852], then as in 2D.
 *
 * Threading: a surrogate object is used by one host thread at a time; its
 * calls are stream-ordered, and work of two calls on one object must not
 * overlap on the GPU.
 */
#ifndef PCSIR_SURROGATE_H_
#define PCSIR_SURROGATE_H_

#include "pcsir.h"
#include "pcsir3.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PCSIR_SUR_PATCH 21
#define PCSIR_SUR_INPUTS 445
#define PCSIR_SUR_HIDDEN 256
#define PCSIR_SUR_NPARAMS (256 * 445 + 256 + 256 * 256 + 256 + 256 + 1)
#define PCSIR_SUR3_PATCH_XY 11
#define PCSIR_SUR3_PATCH_Z 7
#define PCSIR_SUR3_INPUTS 852
#define PCSIR_SUR3_NPARAMS (256 * 852 + 256 + 256 * 256 + 256 + 256 + 1)

typedef struct pcsir_surrogate pcsir_surrogate;

typedef struct pcsir_surrogate_config {
  int64_t capacity;    /* training rows the dataset holds (>= 1) */
  int32_t batch;       /* training minibatch rows: a multiple of 128 in [128, 65536] */
  int32_t geometry;    /* 0 or 2: the 2D surrogate (21 x 21 patch); 3: the 3D one (11 x 11 x 7) */
  double i0_ref;       /* input scale of patch values and of I0 (> 0); a power of two keeps
                          integer photon counts up to 256 + bg exact in bf16 */
  double sigma_ref;    /* input scale of the PSF width (> 0) */
  int64_t max_pixels;  /* largest image (W * H) or volume (W * H * D) the surrogate sees (>= 1) */
} pcsir_surrogate_config;

/* Statistics of the last surrogate-assisted pcSIR step (see
   pcsir_attach_surrogate). */
typedef struct pcsir_surrogate_check {
  int64_t n_dummies;      /* occupied cells of the step */
  int64_t n_exact;        /* dummies whose likelihood was evaluated exactly (held out, clipped, fallback) */
  int64_t n_holdout;      /* held-out dummies checked */
  int64_t n_significant;  /* held-out dummies within the window of the maximum */
  int64_t n_clipped;      /* dummies whose patch leaves the image (always exact) */
  double max_abs_err;     /* largest |predicted - exact| log-likelihood over the significant held-out dummies */
  double rms_err;         /* root mean square of that error over all held-out dummies */
  int32_t fallback;       /* 1: the step used the exact likelihood for every dummy */
  int32_t reserved;
} pcsir_surrogate_check;

/* Creates a surrogate (weights, Adam moments, dataset of capacity rows, and
   the minibatch buffers) on the current device.  The weights start at zero:
   call pcsir_surrogate_init or pcsir_surrogate_set_params.  Errors:
   PCSIR_EINVAL, PCSIR_ENOMEM, PCSIR_ECUDA. */
pcsir_status pcsir_surrogate_create(const pcsir_surrogate_config* cfg, pcsir_surrogate** out);
pcsir_status pcsir_surrogate_destroy(pcsir_surrogate* sur);
const char* pcsir_surrogate_last_error(pcsir_surrogate* sur);

/* Random initial weights on the device (uniform in +-sqrt(3 / fan_in),
   biases 0, from a counter-based hash of seed), zero Adam moments, label
   mean 0 and scale 1. */
pcsir_status pcsir_surrogate_init(pcsir_surrogate* sur, uint64_t seed, void* stream);

/* Host copies of the packed parameters and the label normalisation; both
   calls synchronise the device.  set_params also zeroes the Adam moments. */
pcsir_status pcsir_surrogate_set_params(pcsir_surrogate* sur, const float* params, double label_mean,
                                        double label_scale);
pcsir_status pcsir_surrogate_get_params(pcsir_surrogate* sur, float* params, double* label_mean,
                                        double* label_scale);

/* Appends training rows: the inputs of n states (device double arrays
   x = dummy[0 * stride + i], y = dummy[1 * stride + i], I0 = dummy[4 * stride
   + i], the layout of pcsir_outputs.dummy) against a device image, with
   labels from their exact log-likelihoods ll (device double), the
   background bg and the PSF width psf_sigma.  The stored label is the
   residual ll - T(cx, cy).  A row whose ll lies below label_floor is stored
   "censored", with label label_floor - T: training then only keeps its
   prediction from rising above the floor (censored regression).  A floor some tens of nats below the step's largest
   log-likelihood spares the network the exact values of dummies whose weight
   is negligible anyway (-INFINITY keeps every label exact).  Clipped states
   and rows past the capacity are skipped; pcsir_surrogate_rows reports the
   count. */
pcsir_status pcsir_surrogate_add(pcsir_surrogate* sur, const double* dummy, int64_t stride, int64_t n,
                                 const double* ll, double label_floor, const float* image, int32_t W, int32_t H,
                                 double bg, double psf_sigma, void* stream);

/* The same for a 3D surrogate (geometry 3): states of the 3D step (x =
   dummy[0 * stride + i], y = dummy[1 * stride + i], z = dummy[2 * stride + i],
   I0 = dummy[6 * stride + i], the layout of pcsir3_outputs.dummy) against a
   device volume (D x H x W float32), with the lateral PSF width
   psf_sigma_xy.  Each call accepts the other geometry's surrogate with
   PCSIR_EINVAL only. */
pcsir_status pcsir_surrogate_add3(pcsir_surrogate* sur, const double* dummy, int64_t stride, int64_t n,
                                  const double* ll, double label_floor, const float* volume, int32_t W, int32_t H,
                                  int32_t D, double bg, double psf_sigma_xy, void* stream);

/* Number of packed parameters: PCSIR_SUR_NPARAMS (2D) or PCSIR_SUR3_NPARAMS (3D). */
pcsir_status pcsir_surrogate_nparams(pcsir_surrogate* sur, int64_t* nparams);

/* Rows in the dataset (synchronises the device). */
pcsir_status pcsir_surrogate_rows(pcsir_surrogate* sur, int64_t* rows);
/* Empties the dataset (stream-ordered). */
pcsir_status pcsir_surrogate_clear(pcsir_surrogate* sur, void* stream);

/* Device pointers to the dataset: inputs as bf16 (uint16_t) rows of 448
   values (445 inputs, then 3 zeros; 3D: 896 values, 852 inputs then zeros),
   float32 labels and per-row censoring flags (1: the label is a floor). */
pcsir_status pcsir_surrogate_dataset(pcsir_surrogate* sur, const uint16_t** inputs, const float** labels,
                                     const uint8_t** censored);

/* Label mean and standard deviation of rows [begin, end) become the label
   normalisation (synchronises the device). */
pcsir_status pcsir_surrogate_fit_scale(pcsir_surrogate* sur, int64_t begin, int64_t end);

/* steps Adam updates (learning rate lr, beta1 0.9, beta2 0.999, eps 1e-8) on
   minibatches of cfg.batch rows drawn from [begin, end): with seed != 0 each
   row index is a splitmix64 hash of (seed, update, row) modulo the range;
   with seed == 0 rows are taken in order, cyclically.  The loss is the mean
   over the minibatch of d^2, d = prediction - label in normalised units (0
   for a censored row predicted below its floor); loss (device float array of
   steps entries, or NULL) receives each minibatch's loss before its update. */
pcsir_status pcsir_surrogate_train(pcsir_surrogate* sur, int64_t begin, int64_t end, int32_t steps, double lr,
                                   uint64_t seed, float* loss, void* stream);

/* Gradient of the mean squared error over rows [begin, begin + n) (n a
   multiple of 128, at most cfg.batch) with respect to the packed parameters,
   without an update; grads is a host float array of the packed parameters, loss
   a host double.  Synchronises the device. */
pcsir_status pcsir_surrogate_grads(pcsir_surrogate* sur, int64_t begin, int32_t n, float* grads, double* loss);

/* Predictions of dataset rows [begin, end) in label units (the residual
   label_mean + label_scale * out, without the window term) into out (device
   double array of end - begin). */
pcsir_status pcsir_surrogate_predict_rows(pcsir_surrogate* sur, int64_t begin, int64_t end, double* out,
                                          void* stream);

/* Predicted log-likelihoods of n states (layout as pcsir_surrogate_add)
   into out (device double array of n); clipped states give NaN. */
pcsir_status pcsir_surrogate_predict(pcsir_surrogate* sur, const double* dummy, int64_t stride, int64_t n,
                                     const float* image, int32_t W, int32_t H, double bg, double psf_sigma,
                                     double* out, void* stream);

pcsir_status pcsir_surrogate_predict3(pcsir_surrogate* sur, const double* dummy, int64_t stride, int64_t n,
                                      const float* volume, int32_t W, int32_t H, int32_t D, double bg,
                                      double psf_sigma_xy, double* out, void* stream);

/* Makes pcsir_step on ctx use the surrogate for the dummies' log-likelihoods
   (sur == NULL detaches).  Every step then evaluates the exact likelihood
   only for clipped dummies and for held-out dummies: a cell (bx, by) is held
   out when the top 24 bits of splitmix64(key + salt * 0x9E3779B97F4A7C15),
   key = (uint32)bx | (uint64)(uint32)by << 32, fall below
   floor(f * 2^24) with f = max(holdout_frac, min_holdout / n_dummies) and
   salt the number of earlier steps of ctx since the attach.  A held-out
   dummy is significant when its exact or predicted log-likelihood lies
   within window of the step's largest; when the largest error over the
   significant held-out dummies exceeds max_err (or is not finite) the step
   evaluates the exact likelihood for every dummy, which gives the result of
   the plain step.  Requires a context with patch 21 and the Poisson
   likelihood, and images of at most max_pixels; the surrogate must outlive
   the attachment.  Errors:
   PCSIR_EINVAL, PCSIR_ENOMEM, PCSIR_ECUDA. */
pcsir_status pcsir_attach_surrogate(pcsir_ctx* ctx, pcsir_surrogate* sur, double holdout_frac, int32_t min_holdout,
                                    double window, double max_err);

/* Statistics of the last surrogate-assisted step of ctx (synchronises). */
pcsir_status pcsir_surrogate_last_check(pcsir_ctx* ctx, pcsir_surrogate_check* out);

/* The same for the 3D step (pcsir3_step) with a 3D surrogate: a cell (bx, by,
   bz) is held out by the rule above with key = (bx + 2^20) | (by + 2^20) << 21
   | (bz + 2^20) << 42; requires a context with an 11 x 11 x 7 patch and
   volumes of at most max_pixels voxels. */
pcsir_status pcsir3_attach_surrogate(pcsir3_ctx* ctx, pcsir_surrogate* sur, double holdout_frac,
                                     int32_t min_holdout, double window, double max_err);
pcsir_status pcsir3_surrogate_last_check(pcsir3_ctx* ctx, pcsir_surrogate_check* out);

#ifdef __cplusplus
}
#endif

#endif /* PCSIR_SURROGATE_H_ */
