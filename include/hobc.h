/*
 * hobc.h -- C ABI of the GB300 library for spectral Tikhonov deblurring under
 * high-order (polynomial-preserving) boundary conditions, with the
 * regularisation parameter chosen by generalized cross validation (GCV).
 *
 * Method: M. Donatelli, "Fast transforms for high order boundary conditions"
 * (arXiv:0906.2704).  Section and equation references below use the paper's
 * equation labels, e.g. Eq. (eq:Tc).
 *
 * Problem statement (Sec. 1, Eq. (eq:mod_cont); Sec. 4, Eq. (eq:mintik)):
 *   observed signal or image g (n or n0 x n1 samples), PSF mask h of odd size
 *   centred on its middle entry (g_i = sum_j h_j f_{i-j}), boundary condition of
 *   polynomial degree 1 or 2, smoothing operator L (identity or Laplacian) and a
 *   grid of regularisation parameters mu_0..mu_{K-1} > 0.  The library returns
 *   f_reg = T_X Phi D^{-1} T_X^{-1} g at mu* = argmin_j G(mu_j)
 *   (Eq. (eq:freg), (eq:mugcv)), the index of mu*, and optionally G(mu_j).
 *
 * Conventions shared by every call:
 *   - All device pointers are caller-owned CUDA device memory on the plan's
 *     device; host pointers are caller-owned host memory (pinned memory gives
 *     asynchronous copies).  The library never frees a caller buffer.
 *   - Real arrays are row-major, element type double (HOBC_FP64) or float
 *     (HOBC_FP32).  A batch of `batch` problems is stored back to back.
 *   - Every call is asynchronous on the plan's stream unless stated otherwise;
 *     errors are returned as hobc_status and never thrown across the ABI.
 *   - The plan owns its workspace (allocated once in hobc_plan_create) and its
 *     tables; one plan must not be used from two host threads at once.
 *
 * Spectrum layout (the output of hobc_analysis, the input of hobc_synthesis,
 * and the layout of hobc_eigenvalues):  spectral index t of one axis is column
 * t of T_X on that axis: t = 0 is the left border vector (p or q), t = 1..n-2
 * the trigonometric columns in the natural order of the transform, t = n-1 the
 * right border vector.  SINE_CUBIC, COSINE_QUARTIC and FOURIER_QUARTIC have two
 * border columns on each side: t = 0, 1 (L1, L2 or Q1, Q2) and t = n-2, n-1
 * (their flips), t = 2..n-3 trigonometric.  PERIODIC on the FFT path has none:
 * t = 0..n-1 are the DFT frequencies.
 *   Families SINE, SINE_CUBIC, COSINE and COSINE_QUARTIC keep real spectra: one item is n values (1D) or
 *   n1 x n0 values stored as [t1][t0] (2D, t0 fastest).
 *   Family FOURIER stores complex values (re, im interleaved) and, because g is
 *   real, only the half of axis 1 that determines the rest:
 *   W = floor((n-2)/2) + 3 entries, index c = 0 -> t = 0, c = 1..W-2 -> t = c
 *   (frequencies 0..floor((n-2)/2)), c = W-1 -> t = n-1.  One item is W values
 *   (1D) or W1 x n0 values stored as [c][t0] (2D).  FOURIER_QUARTIC stores the
 *   same way with W = floor((n-4)/2) + 5 (c = 0, 1 -> t = 0, 1; c = W-2, W-1 ->
 *   t = n-2, n-1), PERIODIC with W = floor(n/2) + 1 (c = t).  hobc_spectrum_size
 *   reports the per-item element counts.
 */
#ifndef HOBC_H
#define HOBC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HOBC_OK = 0,
    HOBC_ERR_ARG = 1,          /* null pointer, bad enum, bad size, mu <= 0            */
    HOBC_ERR_UNSUPPORTED = 2,  /* combination the paper gives no fast algorithm for    */
    HOBC_ERR_SIZE = 3,         /* PSF too large for the field of view, n out of range  */
    HOBC_ERR_NONFINITE = 4,    /* non-finite value in the mu grid                      */
    HOBC_ERR_CUDA = 5,         /* a CUDA runtime call failed; see hobc_last_error      */
    HOBC_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up                   */
} hobc_status;

typedef enum {
    HOBC_FAMILY_AUTO = 0,      /* degree 1 -> SINE; degree 2 -> COSINE if the desc says
                                  the PSF is symmetric, else FOURIER; degree 3 -> SINE_CUBIC;
                                  degree 4 -> COSINE_QUARTIC if symmetric, else
                                  FOURIER_QUARTIC                                          */
    HOBC_FAMILY_SINE = 1,      /* antireflective, Sec. 2.2, Eq. (eq:ART), (eq:jcf)       */
    HOBC_FAMILY_COSINE = 2,    /* degree 2, symmetric PSF, Sec. 3.1, Eq. (eq:Tc), (eq:Ac) */
    HOBC_FAMILY_FOURIER = 3,   /* degree 2, any PSF, Sec. 3.2, Eq. (eq:Tf), (eq:Af)      */
    HOBC_FAMILY_SINE_CUBIC = 4, /* degree 3, symmetric PSF: DST-I of order n-4 with four
                                  border columns spanning the cubics (the paper names
                                  degree 3 in Sec. 1 and Sec. 7 without a construction) */
    HOBC_FAMILY_REFLECTIVE = 5, /* classical reflective conditions (Sec. 2, Eq. (eq:refm)):
                                  T = C^T, the orthonormal DCT-II of order n, theta_k =
                                  k pi / n; bc_degree 0, symmetric PSF, HOBC_SPLIT_BF16 only */
    HOBC_FAMILY_PERIODIC = 6,   /* classical periodic conditions (Sec. 2, Eq. (eq:permat)),
                                  theta_k = 2 pi k / n, bc_degree 0.  FP64 / FP32: T = F^H,
                                  the unitary DFT of order n on the FFT path (no border
                                  columns), any PSF, complex spectrum stored like FOURIER's
                                  without border entries (a half of floor(n/2)+1 entries on
                                  the last axis); plain method, steps, host calls and the
                                  allocation-free scan.  HOBC_SPLIT_BF16: the real Hartley
                                  basis (for a symmetric PSF it diagonalises the circulant
                                  as F^H does), symmetric PSF only                        */
    HOBC_FAMILY_COSINE_QUARTIC = 7, /* degree 4, symmetric PSF: the construction of Sec. 3.1
                                  with two border columns per side, DCT-II of order n-4 on
                                  x_a = (2a-3) pi/(2(n-4)), border columns (b-x)^2, (b-x)^4
                                  and their flips spanning the quartics with the constant;
                                  the paper names higher orders in Sec. 7 without a
                                  construction.  cond(T) grows like n^3.5 (1e8 at n = 256):
                                  FP32 is meaningful only for small n.  Plain method
                                  (plans, steps, host call, binned / refined / learned mu)
                                  and the exact GCV; not in the dense, batched or 3D paths */
    HOBC_FAMILY_FOURIER_QUARTIC = 8 /* degree 4, any PSF (reading R17): the construction of
                                  Sec. 3.2 with two border columns per side, DFT of order
                                  N = n-4 on x_a = (a-2) 2 pi/N (rows 0, 1 repeat rows n-4,
                                  n-3 and rows n-2, n-1 repeat rows 2, 3), border columns
                                  (b-x)^2, (b-x)^4 and their flips; the quartic-preserving
                                  (and so also cubic-preserving) answer for a nonsymmetric
                                  PSF.  Stored like FOURIER with two border entries on each
                                  side (W = floor(N/2)+5 on the last axis).  FP64 only; plain
                                  method, steps, host calls and the allocation-free scan   */
} hobc_family;

typedef enum {
    HOBC_L_IDENTITY = 0,       /* L = I                                                   */
    HOBC_L_LAPLACIAN = 1       /* L_X = T_X diag(2 - 2cos theta) T_X^{-1} (Sec. 4, Eq. (eq:L));
                                  2D: Kronecker sum, eigenvalue s(t0) + s(t1)             */
} hobc_smoothing;

typedef enum {
    HOBC_FP64 = 0,             /* all arithmetic and I/O in double                        */
    HOBC_FP32 = 1,             /* transforms, filter and GCV terms in float; boundary 2x2
                                  solve, eigenvalues and GCV sums in double; float I/O     */
    HOBC_SPLIT_BF16 = 2        /* SINE, COSINE, SINE_CUBIC, FOURIER and the comparison
                                  families: every transform pass is a dense product with
                                  T_X or T_X^{-1} on the tensor cores, operands split into
                                  bf16 hi/lo, FP32 accumulation (include/hobc_tc.h); the
                                  Fourier family's complex products run as real products
                                  on (re, im) pairs; eigenvalues, filter and GCV as FP32;
                                  float I/O                                               */
} hobc_precision;

typedef struct {
    int ndim;                  /* 1 (signals) or 2 (images)                               */
    int n[2];                  /* field of view: 1D n[0]; 2D n[0] rows x n[1] columns;
                                  each in [6, 1024]                                        */
    int psf[2];                /* PSF mask size (odd): 1D psf[0] = 2m+1; 2D rows x cols;
                                  needs psf[i] <= n[i] - 2 (Sec. 2.2, Sec. 3), or
                                  psf[i] <= n[i] - 4 (and n[i] >= 8) for SINE_CUBIC,
                                  COSINE_QUARTIC and FOURIER_QUARTIC                      */
    int bc_degree;             /* 1, 2, 3 or 4 (0 with the REFLECTIVE / PERIODIC families) */
    hobc_family family;
    int psf_symmetric;         /* caller asserts h_{-j} = h_j on every axis (used by AUTO) */
    hobc_smoothing L;
    hobc_precision prec;
    int n_mu;                  /* K >= 1 grid points                                       */
    int batch;                 /* problems per call, >= 1 (2D: <= 65535)                   */
    int psf_per_item;          /* 0: one PSF for the whole batch; 1: one PSF per problem   */
} hobc_plan_desc;

typedef struct hobc_plan_s hobc_plan;

/* Create a plan.  desc: problem description (copied).  mu_grid_host: K positive
 * finite doubles (copied); FP32 plans need every mu in [1e-18, 1e18].  cuda_stream: a cudaStream_t on the current device,
 * or NULL for the legacy default stream.  Allocates the plan's device workspace
 * and tables (cudaMalloc); synchronous.  On error *out is set to NULL. */
hobc_status hobc_plan_create(const hobc_plan_desc* desc, const double* mu_grid_host,
                             void* cuda_stream, hobc_plan** out);

/* Release the plan and its device memory (synchronises the plan's stream). */
void hobc_plan_destroy(hobc_plan* plan);

/* The resolved family (HOBC_FAMILY_SINE/COSINE/FOURIER) of a plan. */
hobc_family hobc_plan_family(const hobc_plan* plan);

/* Per-item element counts: *spec = values in one item's spectrum (complex
 * values counted once), *spec_is_complex = 1 for FOURIER, *psf = values in one
 * PSF.  Any output pointer may be NULL. */
hobc_status hobc_spectrum_size(const hobc_plan* plan, size_t* spec, int* spec_is_complex,
                               size_t* psf);

/* The whole method on `batch` problems (Sec. 4, Sec. 6):
 *   g_dev   [batch][n...] real input; psf_dev one PSF or [batch] PSFs, row-major;
 *   f_dev   [batch][n...] real output (may not alias g_dev);
 *   mu_index_dev  [batch] int output: grid index of mu* (nullable);
 *   gcv_dev [batch][K] double output: G(mu_j) of Eq. (eq:mugcv) (nullable).
 * Ties in G take the smallest index; NaN values of G never win. */
hobc_status hobc_deblur(hobc_plan* plan, const void* g_dev, const void* psf_dev, void* f_dev,
                        int* mu_index_dev, double* gcv_dev);

/* hobc_deblur with HOST buffers: copies g and the PSF(s) to the plan's
 * workspace, runs the method, copies f (and mu index, G if non-NULL) back, and
 * returns when all of it has finished (hobc_deblur_host_async followed by
 * hobc_plan_wait).  The batch runs as up to four chunks: their uploads back to
 * back on an internal stream, each chunk's kernels on the plan's stream once
 * its upload is done, each download on a second internal stream once its
 * kernels are done (streams created on the first call), so the copies overlap
 * the kernels of other chunks; copies overlap only when g_host and f_host are
 * page-locked.  The PSF is staged through page-locked memory the plan owns. */
hobc_status hobc_deblur_host(hobc_plan* plan, const void* g_host, const void* psf_host,
                             void* f_host, int* mu_index_host, double* gcv_host);

/* Chunks of the host-buffer pipeline of hobc_deblur_host / hobc_deblur_host_async:
 * the batch is cut into `chunks` (1..8; 0 restores the default, 4) whose uploads,
 * kernels and downloads overlap.  More chunks hide more of the first upload and
 * the last download, fewer keep the kernels' grids large.  HOBC_ERR_ARG outside
 * 0..8.  Waits for the plan's queued work first (consecutive host calls are
 * ordered chunk by chunk), so call it between calls, not inside stream capture. */
hobc_status hobc_plan_set_host_chunks(hobc_plan* plan, int chunks);

/* hobc_deblur_host without the final wait: queues the copies and kernels and
 * returns once the PSF has been read (it is copied into the plan's staging).
 * g_host must stay unchanged and f_host, mu_index_host, gcv_host unread until
 * hobc_plan_wait returns; with page-locked buffers the host returns at once.
 * All four host buffers must be page-locked for that: mu_index_host and
 * gcv_host are copied on the plan's stream, and a copy into pageable memory
 * makes the host wait for every kernel queued before it (pass NULL for them, or
 * page-locked buffers, to keep the call asynchronous).
 * Consecutive calls on one plan overlap: a call's uploads run while the
 * previous call's kernels do, each chunk's upload waiting only until the
 * previous call's analysis has read that chunk's input slots, and each chunk's
 * filter + synthesis until the previous call's download has read its output
 * slots (per-chunk events; the small outputs are copied on the plan's stream).
 * No other call may use the plan until hobc_plan_wait.  Errors of the queueing
 * are returned here, errors of the work by hobc_plan_wait. */
hobc_status hobc_deblur_host_async(hobc_plan* plan, const void* g_host, const void* psf_host,
                                   void* f_host, int* mu_index_host, double* gcv_host);

/* Waits until every copy and kernel queued on the plan (its stream and the two
 * host-call streams) has finished.  HOBC_ERR_CUDA if any of it failed. */
hobc_status hobc_plan_wait(hobc_plan* plan);

/* Step: analysis transform ghat = T_X^{-1} g (Thm. 1 / Eq. (eq:Tx); 2D: tensor
 * product, Sec. 6), the boundary-polynomial correction included.
 * g_dev [batch][n...] real; ghat_dev [batch][spectrum] in the spectrum layout. */
hobc_status hobc_analysis(hobc_plan* plan, const void* g_dev, void* ghat_dev);

/* Step: synthesis y = T_X c (Eq. (eq:ART), (eq:Tc), (eq:Tf); 2D tensor product),
 * the polynomial add-back included.  c_dev in the spectrum layout (FOURIER:
 * must be the half of a spectrum with the symmetry of a real image);
 * y_dev [batch][n...] real. */
hobc_status hobc_synthesis(hobc_plan* plan, const void* c_dev, void* y_dev);

/* Step: eigenvalues d_t = z(-theta_t) of A_X (Eq. (eq:symbol), (eq:jcf),
 * (eq:Ac), (eq:Af); 2D: the three-step rule of Sec. 6, i.e. z at the tensor
 * grid with border indices at angle 0), in the spectrum layout, one per PSF
 * (npsf = batch if psf_per_item else 1).  Element type: the plan's precision,
 * complex for FOURIER. */
hobc_status hobc_eigenvalues(hobc_plan* plan, const void* psf_dev, void* d_dev);

/* Step: GCV scan (Eq. (eq:gcv2), (eq:mugcv)): for every problem and every mu_j,
 * G = sum |sigma_i ghat_i|^2 / (sum sigma_i)^2, sigma_i = |s_i|^2/(|d_i|^2 + mu_j |s_i|^2),
 * sums in double; then mu* = argmin.  ghat_dev as from hobc_analysis, d_dev as
 * from hobc_eigenvalues.  gcv_dev [batch][K] (nullable), mu_index_dev [batch]. */
hobc_status hobc_gcv(hobc_plan* plan, const void* ghat_dev, const void* d_dev,
                     double* gcv_dev, int* mu_index_dev);

/* How hobc_gcv and hobc_deblur (and the host calls) evaluate the curve of
 * Eq. (eq:gcv2).  DIRECT (every plan's default): every (entry, mu_j) term, as
 * described above.  EXPANSION: the same G(mu_j) for every grid value through
 * per-bin moments of the entries: a = |d|^2/|s|^2 is grouped in 256 bins
 * uniform in log a over [1e-3 mu_min, 1e3 mu_max) plus one bin below and one
 * above; in a bin of centre abar, 1/(a+mu)^k is expanded in powers of
 * (a - abar)/(abar + mu) up to the 7th, so a bin contributes through 8 moments
 * of e = w|ghat|^2 and 8 of w, and the curve costs bins x K evaluations instead
 * of entries x K.  The series' truncation changes each term by a relative
 * 9 U^8/(1-U)^2 at most (U = sqrt(r) - 1, r the bins' ratio: 3.3e-9 for a grid
 * [1e-8, 1]; hobc_gcv_expansion_bound); the moments are FP32 over pieces of at
 * most 256 entries and FP64 over the pieces, the curve FP32 per bin with
 * float-float sums over the bins.  Deterministic (fixed summation orders).
 * Offered for FP32 and split-BF16 2D plans with one PSF for the batch
 * (HOBC_ERR_UNSUPPORTED otherwise, or when the grid spans so many decades that
 * the bound would exceed 1e-8).  Setting EXPANSION allocates its workspace
 * (about 32 bytes per stored entry plus 32 bytes per 256 entries per problem)
 * and copies the grid to the host once: call it outside stream capture.
 * hobc_gcv_noalloc and the binned, refined, learned and exact choices are not
 * affected. */
typedef enum {
    HOBC_GCV_DIRECT = 0,
    HOBC_GCV_EXPANSION = 1
} hobc_gcv_mode;
hobc_status hobc_plan_set_gcv_mode(hobc_plan* plan, int mode);
/* The plan's mode (-1 for a NULL plan). */
int hobc_plan_gcv_mode(const hobc_plan* plan);
/* The expansion's truncation bound for the plan's grid (relative, per term),
 * or -1 if the mode was never set. */
double hobc_gcv_expansion_bound(const hobc_plan* plan);

/* Step: filter at mu* and synthesis, f = T_X diag(conj(d)/(|d|^2 + mu*|s|^2)) ghat
 * (Eq. (eq:freg)).  mu_index_dev [batch] grid indices. */
hobc_status hobc_filter_synthesis(hobc_plan* plan, const void* ghat_dev, const void* d_dev,
                                  const int* mu_index_dev, void* f_dev);

/* The GCV scan of hobc_gcv for callers that cannot allocate device memory.
 * The paper has no counterpart: this entry point exists for the deployment
 * side only.  Some callers may not call cudaMalloc at all -- code that runs
 * under a memory allocator it does not own (another framework's device pool,
 * a host application that fixes the device-memory budget at start-up), or a
 * latency-critical path that cannot take cudaMalloc's device-wide
 * synchronisation -- and so cannot create a plan.  This call needs no plan and
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   desc: geometry of the problems (ndim, n, family or bc_degree +
 *         psf_symmetric, L, prec, n_mu, batch, psf_per_item; psf is ignored);
 *   ghat_dev, d_dev: spectra and eigenvalues in the spectrum layout, as
 *         hobc_analysis and hobc_eigenvalues produce them;
 *   mu_dev: the K grid values (double, device; FP32: each in [1e-18, 1e18],
 *         not checked here because they live on the device);
 *   gcv_dev: [batch][K] output (nullable); mu_index_dev: [batch] output;
 *   cuda_stream: the stream to run on (NULL: legacy default stream).
 * It runs the kernels hobc_gcv runs, with the same chunking, so its results
 * equal hobc_gcv's bit for bit.  The per-CTA partial sums and the grid's
 * working-precision copy live in one statically allocated device array of
 * hobc_gcv_noalloc_max_bytes() bytes (16 MiB) that every GPU loading the
 * library holds until the process exits (1D problems with K <= 256 in FP32,
 * K <= 128 in FP64 need only the grid there: one thread group sums each
 * problem's whole spectrum).  A request that needs more --
 * batch * ceil(spectrum/chunk) * 2 * K doubles plus the grid -- is rejected
 * with HOBC_ERR_SIZE and a message in hobc_last_error().  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current, and keeps it with the id of the device's context; the
 * first call after that context was destroyed (cudaDeviceReset) looks it up
 * again in the new one.  Make such a first call before any stream capture.
 * The description is checked as hobc_plan_create checks it (psf ignored);
 * HOBC_SPLIT_BF16 and the REFLECTIVE / PERIODIC families are rejected
 * (HOBC_ERR_UNSUPPORTED): their spectra come from the dense engine.
 * All calls share the one array and it keeps the last call's contents; every
 * entry a call reads is written earlier in the same call, so nothing needs
 * clearing, but calls whose work overlaps on the GPU (different streams, or
 * host threads) race on it and must be serialised by the caller. */
hobc_status hobc_gcv_noalloc(const hobc_plan_desc* desc, const void* ghat_dev, const void* d_dev,
                             const double* mu_dev, double* gcv_dev, int* mu_index_dev, void* cuda_stream);

/* Size in bytes of the static scratch array of hobc_gcv_noalloc. */
size_t hobc_gcv_noalloc_max_bytes(void);

/* ---------------------------------------------------------------------------
 * Batches of 2D problems of uneven sizes (Sec. 6 for each problem).
 * Every problem has its own field of view, its own symmetric PSF and its own
 * boundary-condition degree: 1 -> SINE, 2 -> COSINE, 3 -> SINE_CUBIC.  The
 * smoothing operator, precision and mu grid are shared.  Problems are stored
 * back to back: problem i's image occupies elements [img_off[i], img_off[i+1])
 * (n[0] x n[1], row-major) of the packed g and f buffers, its PSF elements
 * [psf_off[i], psf_off[i+1]) of the packed PSF buffer (hobc_batch_offsets).
 * ------------------------------------------------------------------------- */
typedef struct {
    int n[2];                  /* field of view, each in [8, 512] (COSINE: [8, 1024])      */
    int psf[2];                /* odd PSF size, <= n - 2 (SINE_CUBIC: <= n - 4), <= 63     */
    int bc_degree;             /* 1, 2 or 3                                                */
} hobc_batch_item;

typedef struct {
    int count;                 /* number of problems                                       */
    hobc_smoothing L;
    hobc_precision prec;
    int n_mu;                  /* K >= 1 (FP32: every mu in [1e-18, 1e18])                 */
    int gcv_mode;              /* HOBC_GCV_DIRECT (0) or HOBC_GCV_EXPANSION (FP32 batches):
                                  the curve by bin expansion as for plans (the truncation
                                  bound of hobc_plan_set_gcv_mode, HOBC_ERR_UNSUPPORTED when
                                  it would pass 1e-8); each problem's entries are grouped by
                                  key within chunks of 2048 entries, 16 moments per key
                                  present in the key's slot of the chunk's record, added
                                  chunk by chunk per problem.  The records take a fixed
                                  slot per key: 258 x 64 bytes per chunk (about 8 bytes per
                                  spectrum entry) of device memory, allocated here       */
} hobc_batch_desc;

typedef struct hobc_batch_s hobc_batch;

/* Build the batch plan: transform tables once per distinct (family, n), work
 * lists of every pass, workspace.  Every pass is one launch of a persistent
 * kernel for all families: resident CTAs (the SMs times the CTAs that fit on
 * one) take the pass's work items -- (problem, block of lines) for the line
 * transforms, (problem, chunk) for the GCV scan, (problem, column) for the
 * eigenvalues -- from a device counter, costliest first; the counters are
 * zeroed at the head of each call.  With gcv_mode = HOBC_GCV_EXPANSION the GCV
 * pass takes its (problem, chunk) items in a fixed round robin over its CTAs
 * instead (the chunks cost the same), then one CTA per problem forms its curve.  With a non-NULL stream the whole launch
 * sequence is captured once into a CUDA graph that hobc_deblur_batched
 * replays; with the legacy NULL stream the kernels are launched directly.
 * Synchronous; allocates device memory. */
hobc_status hobc_batch_create(const hobc_batch_desc* desc, const hobc_batch_item* items_host,
                              const double* mu_grid_host, void* cuda_stream, hobc_batch** out);

/* The FFT schedule of one kind of line: problems of this boundary-condition
 * degree whose lines need an FFT of length fft_length (hobc_fft_length) run
 * their FFT stages in radix 16 (16 values a thread, fft_length/16 threads a
 * line pair; fft_length >= 256 only, else radix 8) or radix 8 (fft_length/8
 * threads); 0 keeps the default (radix 16 from 256 up).  Tables of these
 * choices are what an autotuner measures (paper_0906_2704_gb300/autotune.py). */
typedef struct {
    int bc_degree;             /* 1, 2 or 3                                                */
    int fft_length;            /* power of two                                             */
    int radix;                 /* 0, 8 or 16                                               */
} hobc_fft_schedule;

/* hobc_batch_create with an FFT schedule (schedule_len entries, copied; kinds
 * of line it does not list keep the default).  HOBC_ERR_ARG on a malformed
 * entry. */
hobc_status hobc_batch_create_tuned(const hobc_batch_desc* desc, const hobc_batch_item* items_host,
                                    const double* mu_grid_host, const hobc_fft_schedule* schedule,
                                    int schedule_len, void* cuda_stream, hobc_batch** out);

/* FFT length of a line of n samples (8 <= n <= 1024) under boundary-condition
 * degree 1, 2 or 3 (0 otherwise): the power of two the transform of that line
 * runs on (N = n - 2, or n - 4 for degree 3; a core DFT of length N, or
 * 2(N + 1) for degrees 1 and 3, padded to 2^k >= 2 L - 1 for the chirp-z form
 * unless it is a power of two itself). */
int hobc_fft_length(int bc_degree, int n);
void hobc_batch_destroy(hobc_batch* batch);

/* Packed-layout offsets (host arrays of count + 1 elements each, nullable). */
hobc_status hobc_batch_offsets(const hobc_batch* batch, size_t* img_off, size_t* psf_off);

/* Kernel launches per batched deblur (one per pass). */
int hobc_batch_launch_count(const hobc_batch* batch);

/* The whole method on every problem of the batch: g_dev, f_dev packed images,
 * psf_dev packed PSFs, mu_index_dev [count] (nullable), gcv_dev [count][K]
 * (nullable).  Asynchronous on the batch's stream. */
hobc_status hobc_deblur_batched(hobc_batch* batch, const void* g_dev, const void* psf_dev, void* f_dev,
                                int* mu_index_dev, double* gcv_dev);

/* Number of kernel launches the last call on this plan issued. */
int hobc_last_launch_count(const hobc_plan* plan);

/* Human-readable name of a status; text of the last CUDA error seen by the
 * library on this host thread (empty if none). */
const char* hobc_status_str(hobc_status s);
const char* hobc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HOBC_H */
