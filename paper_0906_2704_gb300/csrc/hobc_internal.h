// Host-side plan of the library (see include/hobc.h for the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <complex>

#include "../../include/hobc.h"
#include "../../include/hobc_volume.h"
#include "hobc_device.cuh"

namespace hobc {

// One transform axis as built on the host; device tables are in the plan's
// precision (float or double), the eigen-exponential table always in double.
struct AxisHost {
    int fam, n, N, L, M, log2M, blue, tpg, H, W;
    int r16;        // radix-16 FFT stages (else radix 8)
    int sslot;      // stage rows of the pair kernels inside the group's buffer from this slot (-1: apart)
    void* tw;       // [M] complex
    void* chirp;    // [L] complex (Bluestein only)
    void* bhat;     // [M] complex (Bluestein only)
    void* post;     // [N] complex (COSINE only)
    void* q;        // [n] real
    void* q2;       // [n] real, S3, C4, F4 (second border column)
    double ka, kb, q1, sc, s0, s1, is0, is1, invN;
    double k4[16];  // S3, C4, F4: inverse of the 4x4 border system
    int p;          // PSF extent on this axis
    double2* etab;  // [W][p] exp(-i (j - m) theta_t) for the stored entries t
    float4* etab2;  // the same split into float pairs: (re hi, re lo, im hi, im lo)
};

struct Launch {     // grid/block/shared memory of one line-transform kernel
    dim3 grid, block;
    size_t smem;
};

}  // namespace hobc

struct hobc_plan_s {
    hobc_plan_desc desc;
    int fam;                 // resolved family
    int prec;                // HOBC_FP64 / HOBC_FP32
    size_t esz;              // bytes of one real element (8 or 4)
    cudaStream_t stream;
    int device;
    int K;
    double* mu;              // [K] device
    void* muT;               // [K] device, plan precision
    hobc::AxisHost ax[2];    // 1D: ax[0] only; 2D: ax[0] rows (axis 0), ax[1] columns (axis 1)
    int nax;
    size_t spec_elems;       // stored spectral entries per item
    size_t spec_bytes;       // bytes per item (complex entries count twice)
    size_t img_elems;        // real samples per item
    size_t psf_elems;        // values per PSF
    int npsf;
    // workspace
    void* R;                 // [batch][spec] intermediate of the 2D passes
    void* G;                 // [batch][spec] spectrum
    void* D;                 // [npsf][spec] eigenvalues
    double* partials;        // [batch][chunks][2K]
    int gcv_chunk, gcv_chunks;
    double* gcv;             // [batch][K]
    int* mu_idx;             // [batch]
    void* g_in;              // [batch][img] host-call staging
    void* f_out;             // [batch][img]
    void* psf_in;            // [npsf][psf]
    int launches;
    // learned-mu workspace, allocated on first use (hobc_learned.cu)
    double* feat_partials;   // [batch][feature chunks][3 * bins]
    float* feat;             // [batch][2 * bins]
    float* mlp_y;            // [batch] predicted log10(mu)
    void* bracket_mu;        // [batch][J] plan precision
    double* mu_hat;          // [batch]
    int* bracket_k0;         // [batch]
    double* bracket_partials;// [batch][chunks][2J]
    double* bracket_G;       // [batch][J]
    int* bracket_idx;        // [batch]
    double* mu_val;          // [batch] mu* used by the filter
    int* fell_back;          // [batch]
    double* log_grid;        // [K] log10 of the mu grid (host-computed)
    unsigned char* bin_tab;  // [spec] radial bin (bits 0-5) and pair weight flag (bit 6)
    double* ahist_partials;  // [batch][chunks][3][128] histogram over log10 a of the binned choice
    void* a_edges;           // [129] bin edges, plan precision
    int* k_hat;              // [batch] argmin of the binned G
    double* refine_state;    // [batch][4] lo, mid, hi (log10 mu) and the incumbent mu of the refinement
    cudaStream_t aux[2];     // host-buffer pipeline: upload and download streams (created on first use)
    cudaEvent_t ev_up[8];    // per chunk of the host-buffer pipeline: upload done,
    cudaEvent_t ev_an[8];    // analysis done (the chunk's input slots are free again),
    cudaEvent_t ev_done[8];  // kernels done (its output slots are ready),
    cudaEvent_t ev_down[8];  // download done (its output slots are free again)
    cudaEvent_t ev_psf;      // the PSF staging copy of the last host call has reached the device
    void* psf_pinned;        // page-locked host staging of the PSF(s) for the host calls
    int grid_ascending;      // 1 if the mu grid is strictly increasing
    struct hobc_dense_s* dense;   // HOBC_SPLIT_BF16: matrices and operand workspace (hobc_tc.cu)
    struct hobc_exact_s* exact;   // exact GCV: Gram factors and line sums, allocated on first use (hobc_exact.cu)
    size_t item0;            // first problem of this view of the plan (0 for the plan itself)
    int gcv_mode;            // HOBC_GCV_DIRECT / HOBC_GCV_EXPANSION (hobc_plan_set_gcv_mode)
    struct hobc_gcvx_s* gx;  // the expansion's workspace, allocated when the mode is set (hobc_gcvx.cu)
    int gx_prepared;         // views of the host pipeline: the eigenvalue steps of the expansion already ran
    int host_chunks;         // chunks of the host-buffer pipeline (0: the default)
};

// A 3D plan (include/hobc_volume.h): 2D passes over the slices, a transpose
// and a pass along axis 0 (hobc_volume.cu, hobc_volume.cuh).
struct hobc_volume_s {
    hobc_volume_desc desc;
    int fam;                 // resolved family
    int prec;
    size_t esz;              // bytes of one stored spectral entry
    cudaStream_t stream;
    int K, npsf;
    hobc_plan* slice;        // 2D plan of the (n1, n2) slices, batch x n0 problems (its G is a workspace)
    hobc::AxisHost az;       // axis 0: complex lines for the Fourier family
    size_t S2, S3;           // stored entries of a slice and of a volume
    void* X;                 // [batch][S3] axis-0 lines
    void* G;                 // [batch][S3] spectrum (hobc_volume_deblur)
    void* D;                 // [npsf][S3] eigenvalues (hobc_volume_deblur)
    void* D2;                // [npsf p0][S2] eigenvalues of the PSF's slices
    double* partials;        // [batch][chunks][2K]
    int chunk, chunks;
    int* mu_idx;             // [batch]
    int launches;
};

namespace hobc {

template <typename T> hobc_status run_eig(hobc_plan_s* p, const void* psf, void* D);
template <typename T> hobc_status run_analysis(hobc_plan_s* p, const void* g, void* ghat);
template <typename T> hobc_status run_synthesis(hobc_plan_s* p, const void* c, void* y);
template <typename T> hobc_status run_gcv(hobc_plan_s* p, const void* ghat, const void* D, double* gcv,
                                          int* mu_idx);
template <typename T> hobc_status run_filter_synthesis(hobc_plan_s* p, const void* ghat, const void* D,
                                                       const int* mu_idx, void* f);
template <typename T> hobc_status run_filter_synthesis_mu(hobc_plan_s* p, const void* ghat, const void* D,
                                                          const double* mu_val, void* f);
template <typename T> hobc_status prepare_kernels(hobc_plan_s* p);
void free_learned_ws(hobc_plan_s* p);
void gcvx_free(hobc_plan_s* p);
bool gcvx_active(const hobc_plan_s* p);
hobc_status run_gcv_expansion(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx);
hobc_status gcvx_prepare(hobc_plan_s* p, const void* D);
hobc_status dense_prepare(hobc_plan_s* p);
void dense_free(hobc_plan_s* p);
hobc_status dense_analysis(hobc_plan_s* p, const void* g, void* ghat);
hobc_status dense_synthesis(hobc_plan_s* p, const void* c, void* y);
hobc_status dense_filter_synthesis(hobc_plan_s* p, const void* ghat, const void* D, const int* mu_idx,
                                   const double* mu_val, void* f);

// Families run by the plain method alone (plans, steps, host calls, the
// allocation-free scan): periodic on the FFT path and the degree-4 Fourier family.
inline bool plain_only_family(int fam) { return fam == FAM_P || fam == FAM_F4; }

// power-of-two FFT length of a line of n samples of a family (hobc_api.cu)
int fft_length_of(int fam, int n);
// radix: 0 the default (fft_r16), 16 or 8 to choose (16 only where M >= 256 and log2 M <= 12)
template <typename T> cudaError_t build_axis_host(AxisHost& a, int fam, int n, int p, bool half, int radix = 0);
void free_axis(AxisHost& a);
// 3D launch sequences (hobc_volume.cuh); D == nullptr: plain synthesis
template <typename T> hobc_status run3_analysis(hobc_volume_s* q, const void* g, void* ghat);
template <typename T> hobc_status run3_synthesis(hobc_volume_s* q, const void* c, void* y, const void* D,
                                                 const int* mu_idx);
template <typename T> hobc_status run3_eig(hobc_volume_s* q, const void* psf, void* D);
template <typename T> hobc_status run3_gcv(hobc_volume_s* q, const void* ghat, const void* D, double* gcv,
                                           int* mu_idx);
// exp(-i pi a / b) with the argument reduced exactly; theta_t / pi of spectral
// index t of a family's axis as the fraction num / den (hobc_api.cu)
std::complex<double> expm_ipi(long long a, long long b);
void theta_frac(int fam, int n, int t, long long& num, long long& den);
// Checks a plan description (geometry, family, precision; the PSF extents too if
// check_psf) and resolves HOBC_FAMILY_AUTO into *fam (hobc_api.cu).
hobc_status resolve_desc(const hobc_plan_desc& d, bool check_psf, int* fam);
void set_last_error(const char* what, cudaError_t e);
void set_last_error_text(const char* text);
hobc_status launch_gcv_finalize(hobc_plan_s* p, double* gcv, int* mu_idx);
void exact_free(hobc_plan_s* p);
// G(mu_j) and the grid argmin of each problem from its chunk partials: one
// cluster of up to 8 CTAs per problem (hobc_api.cu)
cudaError_t launch_gcv_finalize_raw(const double* partials, int nchunks, int K, int batch, double* gcv,
                                    int* mu_idx, cudaStream_t st);

}  // namespace hobc
