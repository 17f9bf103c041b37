/*
 * The method on 3D arrays (Sec. 6, the multidimensional case): the transform
 * is the tensor product T_X^(3) = T_{X,n0} (x) T_{X,n1} (x) T_{X,n2}, the
 * eigenvalues of the PSF are its 3D symbol z(-theta_t0, -theta_t1,
 * -theta_t2) on the tensor grid, and the Laplacian is the Kronecker sum
 * s(t0) + s(t1) + s(t2).  Everything else (the GCV functional of Eq. (eq:gcv2),
 * (eq:mugcv) and the filter of Eq. (eq:freg)) is per spectral entry, as in 1D
 * and 2D.
 *
 * Layouts.  A volume is [n0][n1][n2] row-major (n2 fastest); a PSF
 * [p0][p1][p2] likewise (odd sizes, centred).  The spectrum of one volume holds
 * S3 = S2 * n0 entries at ((c * n1 + t1) * n0 + t0), with (c, t1) the stored
 * position of the 2D spectrum of an (n1, n2) slice (include/hobc.h: c the
 * stored index along axis 2, a half spectrum for the Fourier family, t1 the
 * index along axis 1) and t0 the spectral index along axis 0, innermost.
 * Entries are complex (re, im pairs) for the Fourier family, real otherwise.
 *
 * Conventions are those of hobc.h: device pointers, calls asynchronous on the
 * plan's stream, errors as hobc_status with hobc_last_error() for CUDA
 * failures.  FP64 and FP32 plans (HOBC_SPLIT_BF16 returns
 * HOBC_ERR_UNSUPPORTED).  Work runs as 2D passes over the batch x n0 slices
 * (batch * n0 <= 65535), a transpose, and a pass along axis 0.
 */
#ifndef HOBC_VOLUME_H
#define HOBC_VOLUME_H

#include "hobc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n[3];                  /* field of view n0 x n1 x n2, each in [6, 1024]          */
    int psf[3];                /* PSF mask p0 x p1 x p2 (odd), p_i <= n_i - 2 (n_i - 4 for
                                  degree 3)                                               */
    int bc_degree;             /* 1, 2 or 3                                                */
    hobc_family family;        /* AUTO, SINE, COSINE, FOURIER or SINE_CUBIC                */
    int psf_symmetric;         /* caller asserts h symmetric on every axis (used by AUTO) */
    hobc_smoothing L;
    hobc_precision prec;       /* HOBC_FP64 or HOBC_FP32                                   */
    int n_mu;
    int batch;                 /* volumes per call                                         */
    int psf_per_item;
} hobc_volume_desc;

typedef struct hobc_volume_s hobc_volume;

/* Create / destroy a 3D plan (mu grid as in hobc_plan_create; synchronous). */
hobc_status hobc_volume_create(const hobc_volume_desc* desc, const double* mu_grid_host, void* cuda_stream,
                               hobc_volume** out);
void hobc_volume_destroy(hobc_volume* plan);

/* Stored spectral entries per volume (S3) and whether they are complex. */
hobc_status hobc_volume_spectrum_size(const hobc_volume* plan, size_t* spec, int* spec_is_complex);

/* Steps, as their 1D / 2D counterparts in hobc.h. */
hobc_status hobc_volume_analysis(hobc_volume* plan, const void* g_dev, void* ghat_dev);
hobc_status hobc_volume_synthesis(hobc_volume* plan, const void* c_dev, void* y_dev);
hobc_status hobc_volume_eigenvalues(hobc_volume* plan, const void* psf_dev, void* d_dev);
hobc_status hobc_volume_gcv(hobc_volume* plan, const void* ghat_dev, const void* d_dev, double* gcv_dev,
                            int* mu_index_dev);
hobc_status hobc_volume_filter_synthesis(hobc_volume* plan, const void* ghat_dev, const void* d_dev,
                                         const int* mu_index_dev, void* f_dev);

/* The whole method on a batch of volumes: eigenvalues, analysis, GCV scan and
 * argmin, filter at mu* and synthesis (mu_index_dev, gcv_dev nullable). */
hobc_status hobc_volume_deblur(hobc_volume* plan, const void* g_dev, const void* psf_dev, void* f_dev,
                               int* mu_index_dev, double* gcv_dev);

/* Kernel launches of the last call on this plan. */
int hobc_volume_launch_count(const hobc_volume* plan);

#ifdef __cplusplus
}
#endif

#endif /* HOBC_VOLUME_H */
