/* Learned surrogate of the intralaminar damage law (Algorithm 4).
 *
 * A multilayer perceptron 10 -> 64 -> 64 -> 64 -> 10 (ReLU, 9,674
 * parameters) maps the elastic strain of a Gauss point (ply axes, engineering
 * shear, after the exact shear plasticity of Algorithm 4) and its four damage
 * thresholds r_FT, r_FC, r_MT, r_MC to the nominal stress and the updated
 * thresholds.  Weights are BF16 with FP32 accumulation on the Blackwell
 * tensor cores (tcgen05.mma with the accumulators in tensor memory, 128
 * points per CTA) in training (forward, backward, weight gradients) and in
 * inference; training keeps FP32 master weights (Adam).  Every wait on the
 * tensor core is bounded: one that gives up returns PDN_E_TIMEOUT from the
 * call (or halts a stepping context with it).
 *
 * Training data come from the library's own exact law on the GPU (the same
 * device code the hex kernel runs, checked against the FP64 CPU law in the
 * tests) along seeded monotonic and cyclic elastic-strain paths from the
 * undamaged state.  Only points in the surrogate's regime are kept: every
 * loading function below onset_ratio times its threshold (so no threshold
 * grows), which is also the regime where the hex kernel uses the network.
 * Elsewhere (near onset, or an input outside the box spanned by the training
 * data) the hex kernel evaluates the exact law.  In that regime the exact
 * thresholds do not change, so the hex kernel keeps them and uses the network
 * for the stress only; the threshold outputs are trained and reported.
 *
 * Inputs and outputs in raw units: strain [11 22 33 12 13 23] (engineering
 * shear), thresholds (>= 1), stress in MPa.  Element-level strength seeding
 * is not an input: the network learns the nominal strengths and one crack-band
 * length lc. */
#ifndef PDN_SURROGATE_H
#define PDN_SURROGATE_H

#include <stdint.h>

#include "pdn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdn_surrogate pdn_surrogate;

#define PDN_SUR_PARAMS 9674 /* W1[64][10], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[10][64], b4[10] */
#define PDN_SUR_SCALING 60  /* in_shift[10], in_mul[10], out_shift[10], out_mul[10], lo[10], hi[10] */

/* Create a surrogate for a material (nominal strengths, spread ignored) and
 * crack-band length lc (mm) on the current device; parameters initialised
 * from seed (He-uniform weights, zero biases), identity scaling.  stream as
 * in pdn_options.  PDN_E_UNSTABLE when lc is at or past the snap-back length
 * 2 E G / X^2 of any mode: there the exact law drops to zero stress at onset,
 * a jump in the thresholds that the network does not represent. */
int pdn_sur_create(pdn_surrogate **out, const pdn_material *mat, double lc, uint64_t seed, void *stream);

/* Training set: n_paths seeded elastic-strain paths of steps_per_path
 * increments each (a fraction cyclic_fraction cyclic, 1 to 3 half-waves;
 * the rest monotonic), components uniform in [-strain_max, strain_max]
 * (shear: twice that) times a path amplitude uniform in (0, 1].  The exact
 * damage law is applied along each path from the undamaged state; points
 * whose largest loading-function ratio phi/r is at most onset_ratio are kept
 * (in path order).  Sets the input/output scaling (mean and spread of the
 * kept points) and the training box.  *n_kept receives their number. */
int pdn_sur_generate(pdn_surrogate *s, int64_t n_paths, int32_t steps_per_path, double strain_max,
                     double cyclic_fraction, double onset_ratio, uint64_t seed, int64_t *n_kept);

/* Copy points [offset, offset + n) of the training set (raw units, x[n][10],
 * y[n][10]; host arrays, either may be NULL). */
int pdn_sur_get_data(pdn_surrogate *s, int64_t offset, int64_t n, float *x, float *y);

/* iters Adam steps (learning rate lr with cosine decay to lr/100) on seeded
 * minibatches of `batch` points (a multiple of 128) drawn from the training
 * set; loss (mean squared error of the normalised outputs) of each step into
 * loss[iters] when not NULL. */
int pdn_sur_train(pdn_surrogate *s, int64_t iters, int32_t batch, double lr, uint64_t seed, double *loss);

/* Network output for n points: in[n][10] raw -> out[n][10] raw.  Pointers
 * are device pointers when on_device != 0. */
int pdn_sur_forward(pdn_surrogate *s, const float *in, float *out, int64_t n, int32_t on_device);

/* The exact damage law (FP64) for the same points, for comparison. */
int pdn_sur_exact(pdn_surrogate *s, const float *in, float *out, int64_t n, int32_t on_device);

/* Gradient of the loss with respect to the parameters (exchange order of
 * PDN_SUR_PARAMS) for n (a multiple of 128) normalised inputs xn[n][10] and
 * normalised targets tn[n][10] (host arrays); *loss receives the loss.  The
 * parameters are not changed. */
int pdn_sur_gradient(pdn_surrogate *s, const float *xn, const float *tn, int64_t n, float *grad, double *loss);

/* FP32 master parameters and scaling (host arrays; either may be NULL). */
int pdn_sur_get_params(pdn_surrogate *s, float *params, float *scaling);
int pdn_sur_set_params(pdn_surrogate *s, const float *params, const float *scaling);

/* Use surrogate s for the intralaminar law of context ctx from its next
 * step (FP32 element mode with axis-aligned box elements; other contexts
 * return PDN_E_ARG): points whose loading-function ratios are all at most
 * onset_ratio and whose inputs lie in the training box take the network's
 * stress, the others the exact law.  s == NULL returns to the exact law.
 * The context copies the parameters: later training of s does not affect it
 * until pdn_set_surrogate is called again. */
int pdn_set_surrogate(pdn_ctx *ctx, pdn_surrogate *s, double onset_ratio);

void pdn_sur_destroy(pdn_surrogate *s);
const char *pdn_sur_last_error(const pdn_surrogate *s);

#ifdef __cplusplus
}
#endif

#endif /* PDN_SURROGATE_H */
