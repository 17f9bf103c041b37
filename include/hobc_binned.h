/*
 * Binned choice of the regularisation parameter: an extension of the method
 * with no counterpart in the paper.  The GCV functional of Eq. (eq:gcv2),
 * (eq:mugcv) depends on a spectral entry only through a = |d|^2/|s|^2 and
 * |ghat|^2:  G(mu) = sum e_i/(a_i + mu)^2 / (sum w_i/(a_i + mu))^2.  Grouping the
 * entries into 128 bins of log10 a between 1e-12 and 1e4 (end bins take
 * everything outside) and replacing a by its bin mean gives G_bin, within a
 * factor r^4 of G for a inside the range (r = 10^(16/128), the bin width).
 * The grid argmin of G_bin only places a bracket; the exact G decides.
 *
 * Conventions are those of hobc.h: device pointers, calls asynchronous on the
 * plan's stream, errors as hobc_status with hobc_last_error() for CUDA
 * failures.  The first call on a plan allocates its workspace for these calls
 * and reads the mu grid back (synchronous); the grid must be strictly
 * increasing (HOBC_ERR_ARG otherwise).
 */
#ifndef HOBC_BINNED_H
#define HOBC_BINNED_H

#include "hobc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Step: the binned choice of mu* on spectra laid out as hobc_analysis /
 * hobc_eigenvalues write them (1D or 2D plans).  Per problem: the histogram
 * (count W, energy E = sum w|ghat|^2 and A = sum w a per bin; w = 2 for a
 * Fourier entry standing for a conjugate pair; entries with s = 0 left out;
 * an entry's bin is the number of interior edges 10^(-12 + b/8) <= a, compared
 * in the plan's precision), G_bin(mu_j) in FP32 with abar = A/W, its first
 * minimiser k_hat (NaN never wins), then the exact G on the min(9, K) grid
 * values around k_hat (shifted inside the grid).  mu* is the first minimiser
 * of that bracket unless it sits on a bracket edge that is not an end of the
 * grid; then the problem falls back to the full grid scan of hobc_gcv.
 * mu_index_dev [batch] receives the grid index of mu*, fell_back_dev [batch]
 * (nullable) 1 where the full scan ran, k_hat_dev [batch] (nullable) k_hat. */
hobc_status hobc_gcv_binned(hobc_plan* plan, const void* ghat_dev, const void* d_dev, int* mu_index_dev,
                            int* fell_back_dev, int* k_hat_dev);

/* The whole method with the binned choice of mu*: as hobc_deblur with
 * hobc_gcv replaced by hobc_gcv_binned (mu_index_dev, fell_back_dev
 * nullable).  Where mu* is the grid minimiser the result equals hobc_deblur's
 * bit for bit. */
hobc_status hobc_deblur_binned(hobc_plan* plan, const void* g_dev, const void* psf_dev, void* f_dev,
                               int* mu_index_dev, int* fell_back_dev);

#ifdef __cplusplus
}
#endif

#endif /* HOBC_BINNED_H */
