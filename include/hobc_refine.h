/*
 * Continuous refinement of the GCV choice of mu.  Eq. (eq:mugcv) defines mu*
 * as the minimiser of the GCV functional of Eq. (eq:gcv2) over all mu > 0; the
 * grid argmin k of hobc_gcv only brackets it.  The refinement searches log10 mu
 * between the grid neighbours mu_{k-1} and mu_{k+1} (clamped to the grid),
 * with the grid value itself as the incumbent: each of 5 rounds evaluates G at
 * nine points (four equal log10 steps from the bracket's low end to the
 * incumbent and four from the incumbent to the high end; the incumbent is
 * re-evaluated), takes the first minimiser (NaN never wins) as the new
 * incumbent and its two neighbours as the new bracket.  A round shrinks the
 * bracket about four times, so mu* is resolved to about 1/1000 of the two grid
 * steps around k.  The evaluation points are values of the plan's precision
 * and G is evaluated as in hobc_gcv (plan-precision terms, FP64 sums).
 *
 * Conventions are those of hobc.h: device pointers, calls asynchronous on the
 * plan's stream, errors as hobc_status with hobc_last_error() for CUDA
 * failures.  The first call on a plan allocates its workspace for these calls
 * (shared with hobc_binned.h and hobc_learned.h) and reads the mu grid back
 * (synchronous); the grid must be strictly increasing (HOBC_ERR_ARG otherwise).
 */
#ifndef HOBC_REFINE_H
#define HOBC_REFINE_H

#include "hobc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Step: the refinement on spectra laid out as hobc_analysis /
 * hobc_eigenvalues write them (1D or 2D plans, every family and precision).
 * mu_index_dev [batch]: the grid argmin of each problem (clamped to the grid),
 * as hobc_gcv writes it.  mu_dev [batch] receives the refined mu* (a value of
 * the plan's precision, stored as double), gcv_dev [batch] (nullable) G at
 * mu*.  16 kernel launches. */
hobc_status hobc_gcv_refine(hobc_plan* plan, const void* ghat_dev, const void* d_dev, const int* mu_index_dev,
                            double* mu_dev, double* gcv_dev);

/* Step: filter and synthesis at per-problem values of mu, f = T_X diag(conj(d)
 * / (|d|^2 + mu |s|^2)) ghat (Eq. (eq:freg)) with mu = mu_dev[item] (double,
 * device; rounded to the plan's precision; FP32 plans need mu in [1e-18, 1e18],
 * which is not checked because the values live on the device). */
hobc_status hobc_filter_synthesis_mu(hobc_plan* plan, const void* ghat_dev, const void* d_dev, const double* mu_dev,
                                     void* f_dev);

/* The whole method with the refined mu*: eigenvalues, analysis, the full GCV
 * grid scan (grid argmin into mu_index_dev, nullable), the refinement (mu*
 * into mu_dev, nullable) and the filter + synthesis at mu*. */
hobc_status hobc_deblur_refined(hobc_plan* plan, const void* g_dev, const void* psf_dev, void* f_dev,
                                int* mu_index_dev, double* mu_dev);

#ifdef __cplusplus
}
#endif

#endif /* HOBC_REFINE_H */
