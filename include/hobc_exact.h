/*
 * The exact GCV functional of Eq. (eq:gcv), as an option beside the paper's
 * approximation (Eq. (eq:gcv2)).  With A = T_X D T_X^{-1} and the reblurred
 * filter of Eq. (eq:freg), g - A f_mu = T_X (I - Phi_mu) ghat, so
 *
 *   G_ex(mu) = ||T_X (sigma . ghat)||^2 / (sum_i sigma_i)^2,
 *   sigma_i = |s_i|^2 / (|d_i|^2 + mu |s_i|^2),
 *
 * the approximate functional with T_X kept in the numerator (both divided by
 * mu^2).  The paper drops T_X because it is close to unitary; it is not
 * for large n (T_C at n = 1024 has condition ~2e4), which is where the two
 * functionals part.  Each axis's T_a is split by rows: the interior rows are
 * X_a^H W_a with X_a^H unitary and W_a = [bhat_L | I | bhat_R] (bhat the
 * transformed interior parts of the k border columns per side), the 2k
 * extension rows are V_a.  In 2D (T = T_0 (x) T_1 acting as T_0 P T_1^T on the
 * spectrum P = sigma . ghat):
 *
 *   ||T P||^2 = ||W0 P W1^T||^2 + ||V0 P W1^T||^2 + ||W0 P V1^T||^2 + ||V0 P V1^T||^2,
 *
 * every term a sum of squares, so rounding is amplified by cond(T), not
 * cond(T)^2.  Per (entry, mu) this costs 1 + 2k reciprocals and about 4k(k+1)
 * products beside the approximation's terms (complex for the Fourier
 * family).  Every family: sine, cosine and Fourier k = 1, degrees 3 and 4 k = 2; the
 * classical reflective and periodic conditions of HOBC_SPLIT_BF16 plans have
 * orthogonal T, k = 0, and G_ex equals the approximation.  The Fourier family
 * stores half of the last axis: a full column of the other half is the
 * conjugate of a stored column with its rows mapped t -> -t, so column sums
 * carry the pair weight 2 and the row sums add the partner entries.
 *
 * Conventions are those of hobc.h: device pointers, calls asynchronous on the
 * plan's stream, errors as hobc_status with hobc_last_error() for CUDA
 * failures.  The first call on a plan builds the row splits (FP64 transforms
 * of the identity, synchronous) and, for 2D plans, allocates the per-line
 * sums (batch x ((3 + 2k c) W_1 + n_0) x K values of the plan's precision;
 * W_1 the stored columns, c = 2 for the Fourier family, else 1).
 */
#ifndef HOBC_EXACT_H
#define HOBC_EXACT_H

#include "hobc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Step: G_ex on every grid value and its first minimiser (NaN never wins),
 * from spectra laid out as hobc_analysis / hobc_eigenvalues write them.
 * gcv_dev [batch][K] (nullable), mu_index_dev [batch].  Sums per line in the
 * plan's precision, across lines in FP64. */
hobc_status hobc_gcv_exact(hobc_plan* plan, const void* ghat_dev, const void* d_dev, double* gcv_dev,
                           int* mu_index_dev);

/* The whole method with mu* chosen by G_ex: eigenvalues, analysis,
 * hobc_gcv_exact, filter + synthesis at the grid value mu*. */
hobc_status hobc_deblur_exact(hobc_plan* plan, const void* g_dev, const void* psf_dev, void* f_dev,
                              int* mu_index_dev, double* gcv_dev);

/* Step: the grid minimiser of G_ex by a coarse-to-fine search over the grid
 * instead of the full scan.  Eq. (eq:mugcv) minimises G over the mu values; the
 * paper evaluates a grid and gives no search.  For 32 < K <= 1921 three levels
 * with s1 = ceil((K - 1) / 15) and s2 = min(s1, max(4, ceil(s1 / 8))): level 0
 * evaluates the grid values 0, s1, 2 s1, ... and K - 1 (at most 16); level 1
 * the incumbent +- s2 m for m = 1 .. ceil(s1 / s2) - 1; level 2 the incumbent
 * +- 1 .. s2 - 1, where the incumbent is the first minimiser (smallest G, then
 * smallest index; NaN never wins) of every value evaluated so far, indices
 * clamped into the grid.  Where G_ex is unimodal over the grid this returns
 * the grid's first minimiser (30 evaluations instead of 256 at K = 256);
 * where it is not, a local minimiser near the best of level 0.  Other K: the
 * full scan of hobc_gcv_exact.
 *   gcv_dev [batch][K] (nullable): G_ex at the evaluated grid values, NaN at
 *   the others; mu_index_dev [batch] the minimiser.  A value may differ from
 *   hobc_gcv_exact's at the same index by rounding (the line sums of a level
 *   with few values are split over several lanes and added in another order). */
hobc_status hobc_gcv_exact_search(hobc_plan* plan, const void* ghat_dev, const void* d_dev, double* gcv_dev,
                                  int* mu_index_dev);

/* hobc_deblur_exact with mu* from hobc_gcv_exact_search. */
hobc_status hobc_deblur_exact_search(hobc_plan* plan, const void* g_dev, const void* psf_dev, void* f_dev,
                                     int* mu_index_dev, double* gcv_dev);

#ifdef __cplusplus
}
#endif

#endif /* HOBC_EXACT_H */
