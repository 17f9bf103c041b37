/*
 * Learned choice of the regularisation parameter: an extension of the method
 * with no counterpart in the paper.  The paper picks mu* by scanning the GCV
 * functional (Eq. (eq:gcv2), (eq:mugcv)) over a grid of K values; here a small
 * network predicts log10(mu*) from two radial spectra of the problem (or from
 * the shares of the GCV terms over log10 a, hobc_features_hist), the GCV
 * functional is evaluated at the prediction and at the nearest grid values
 * only, and a problem whose prediction looks poor falls back to the full scan.
 * The transforms, eigenvalues and filter are the paper's, unchanged.
 *
 * Conventions are those of hobc.h: device pointers unless a name ends in
 * _host, calls asynchronous on the plan's (or network's) stream unless stated,
 * errors reported as hobc_status with hobc_last_error() for CUDA failures.
 */
#ifndef HOBC_LEARNED_H
#define HOBC_LEARNED_H

#include "hobc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Number of radial bins of each spectrum; the network input has 2x this. */
#define HOBC_FEATURE_BINS 64

/* Step: features of every problem of a 2D plan, x_dev [batch][2 * 64] float.
 * Spectral entry (t0, t1) has normalised frequencies f_a = theta_a / pi
 * (border columns 0; FOURIER angles folded into [0, 1] as min(f, 2 - f)) and
 * radius rho = sqrt((f0^2 + f1^2) / 2); its bin is floor(64 rho) (clamped to
 * 63), decided exactly in integer arithmetic.  x[b] = log10(mean |ghat|^2 over
 * bin b + 1e-30), x[64 + b] the same for |d|^2.  ghat_dev, d_dev: the
 * spectrum and eigenvalues as hobc_analysis / hobc_eigenvalues write them.
 * HOBC_ERR_UNSUPPORTED on a 1D plan.  Allocates the plan's learned workspace
 * on first use. */
hobc_status hobc_features(hobc_plan* plan, const void* ghat_dev, const void* d_dev, float* x_dev);

/* Feature kinds the learned path can form (hobc_mlp_set_feature_kind). */
#define HOBC_FEATURES_RADIAL 0     /* hobc_features: radial spectra of |ghat|^2 and |d|^2 (2D plans) */
#define HOBC_FEATURES_HIST 1       /* hobc_features_hist: shares of the GCV terms over log10 a      */

/* Step: histogram features of every problem, x_dev [batch][2 * 64] float.  G
 * of Eq. (eq:gcv2) depends on a spectral entry only through a = |d|^2 / |s|^2
 * and |ghat|^2 (entries with s = 0 drop out), so the features are the shares
 * of those terms over a: the entries are grouped by log10 a into 64 bins of
 * 0.25 decade over [1e-12, 1e4) (values outside go to the end bins; an
 * entry's bin is the number of interior edges 10^(-12 + b / 4) <= a, compared
 * in the plan's precision), and x[b] = log10(E_b / E + 1e-12), x[64 + b] =
 * log10(W_b / W + 1e-12), with E_b the sum of |ghat|^2 and W_b the number of
 * entries in bin b (a stored Fourier entry that stands for a conjugate pair
 * counts twice) and E, W their totals.  1D and 2D plans.  Allocates the plan's
 * learned workspace on first use. */
hobc_status hobc_features_hist(hobc_plan* plan, const void* ghat_dev, const void* d_dev, float* x_dev);

/* ---------------------------------------------------------------------------
 * The network: x (n_in) -> GELU(W1 x' + b1) (n_hidden) -> GELU(W2 h1 + b2)
 * (n_hidden) -> w3 . h2 + b3, x' = (x - mean) / scale per input, GELU(z) =
 * z (1 + erf(z / sqrt 2)) / 2.  FP32 master weights; the three weight matrices
 * are used in BF16 (refreshed after every update), accumulation in FP32.
 * Parameter vector layout (host, float): W1 [n_hidden][n_in], b1 [n_hidden],
 * W2 [n_hidden][n_hidden], b2 [n_hidden], w3 [n_hidden], b3 [1]; set/get take
 * it followed by mean [n_in] and scale [n_in].
 * ------------------------------------------------------------------------- */
typedef struct hobc_mlp_s hobc_mlp;

/* Create a network with zero weights, mean 0, scale 1 (n_in, n_hidden in
 * [1, 4096]).  Synchronous; allocates device memory. */
hobc_status hobc_mlp_create(int n_in, int n_hidden, void* cuda_stream, hobc_mlp** out);
void hobc_mlp_destroy(hobc_mlp* net);

/* Length of the parameter vector (without mean and scale). */
int hobc_mlp_param_count(const hobc_mlp* net);

/* Copy parameters, mean and scale from / to host memory (param_count + 2 n_in
 * floats).  set resets the optimiser moments and step.  Synchronous. */
hobc_status hobc_mlp_set_params(hobc_mlp* net, const float* host);
hobc_status hobc_mlp_get_params(const hobc_mlp* net, float* host);

/* y_dev[b] = network(x_dev[b]) for batch rows of n_in floats. */
hobc_status hobc_mlp_forward(hobc_mlp* net, const float* x_dev, int batch, float* y_dev);

/* Mean squared error against t_dev [batch] and its gradient with respect to
 * every parameter (grad_dev [param_count], nullable; loss_dev [1], nullable). */
hobc_status hobc_mlp_gradients(hobc_mlp* net, const float* x_dev, const float* t_dev, int batch, float* grad_dev,
                               float* loss_dev);

/* One AdamW step (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight decay,
 * bias-corrected moments) on the batch's mean squared error. */
hobc_status hobc_mlp_train_step(hobc_mlp* net, const float* x_dev, const float* t_dev, int batch, float lr,
                                float weight_decay, float* loss_dev);

/* Checkpoint: "HOBCMLP1", int32 n_in, n_hidden, step, param_count; float
 * parameters, mean, scale, first and second moments; uint64 FNV-1a checksum
 * of all preceding bytes.  load rejects a file of another shape or with a bad
 * checksum (HOBC_ERR_ARG).  Synchronous. */
hobc_status hobc_mlp_save(const hobc_mlp* net, const char* path);
hobc_status hobc_mlp_load(hobc_mlp* net, const char* path);

/* Input standardisation from training features: mean[j] and scale[j] =
 * standard deviation + 1e-3 of column j of x_dev [rows][n_in], in FP64 on the
 * GPU (two passes, fixed summation order).  Asynchronous on the network's
 * stream; leaves the weights and optimiser state as they are. */
hobc_status hobc_mlp_fit_scaling(hobc_mlp* net, const float* x_dev, int rows);

/* The features hobc_deblur_learned forms for this network: HOBC_FEATURES_RADIAL
 * (the default on creation) or HOBC_FEATURES_HIST (HOBC_ERR_ARG otherwise).
 * The kind is not part of the checkpoint; set it after hobc_mlp_load.
 * hobc_mlp_feature_kind returns it (-1 for NULL). */
hobc_status hobc_mlp_set_feature_kind(hobc_mlp* net, int kind);
int hobc_mlp_feature_kind(const hobc_mlp* net);

/* Kernel launches of the last forward / gradients / train_step call. */
int hobc_mlp_last_launch_count(const hobc_mlp* net);

/* The whole method on a 2D plan with the learned choice of mu*: eigenvalues,
 * analysis, features, network, then G (Eq. (eq:gcv2)) at the prediction
 * mu_hat (clamped to the grid's range) and at the J - 1 = min(17, K) grid
 * values around it.  mu* = mu_hat unless G(mu_hat) exceeds 1.05 times the
 * smallest of those grid values of G, or that minimum sits on the bracket's
 * edge inside the grid; then that problem falls back to the full grid scan and
 * mu* is its GCV minimiser (lowest index on ties).  Filter and synthesis as
 * hobc_deblur.  mu_dev [batch] (nullable) receives mu*, fell_back_dev [batch]
 * (nullable) 1 where the full scan ran.  The features are those of the
 * network's feature kind.  The network must have n_in = 128
 * (HOBC_ERR_UNSUPPORTED otherwise, and on a 1D plan with radial features); the plan's mu grid must
 * be strictly increasing (HOBC_ERR_ARG otherwise).  The first call on a plan
 * allocates its learned workspace and reads the grid back (synchronous). */
hobc_status hobc_deblur_learned(hobc_plan* plan, hobc_mlp* net, const void* g_dev, const void* psf_dev, void* f_dev,
                                double* mu_dev, int* fell_back_dev);

#ifdef __cplusplus
}
#endif

#endif /* HOBC_LEARNED_H */
