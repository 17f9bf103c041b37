// hobc_gcv_noalloc: the GCV scan (per-CTA partial sums and the argmin) for
// callers that cannot allocate device memory.  The per-CTA partial sums -- the
// only scratch the scan needs -- and the FP32 copy of the mu grid live in one
// file-scope device array instead of a plan's cudaMalloc'd workspace.  The
// kernels are the ones hobc_gcv launches; only where their scratch lives differs.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "hobc_internal.h"
#include "hobc_kernels.cuh"

namespace {

// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_gcv_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};   // device address of g_gcv_scratch, per device

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and kept.
hobc_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { hobc::set_last_error("hobc_gcv_noalloc: cudaGetDevice", e); return HOBC_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return HOBC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gcv_scratch);
        if (e != cudaSuccess) {
            hobc::set_last_error("hobc_gcv_noalloc: cudaGetSymbolAddress", e);
            return HOBC_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HOBC_OK;
}

template <typename T>
__global__ void k_mu_to_working(const double* __restrict__ mu, T* __restrict__ out, int K) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < K; j += gridDim.x * blockDim.x) out[j] = (T)mu[j];
}

template <typename T>
hobc_status launch(const hobc::GcvGeom& geo, int cplx, int batch, int chunks, const void* ghat, const void* d,
                   long long d_psf_stride, int psf_per, const double* mu, unsigned char* scratch,
                   size_t mu_bytes, double* gcv, int* mu_idx, cudaStream_t st) {
    using namespace hobc;
    T* muT = reinterpret_cast<T*>(scratch);
    double* partials = reinterpret_cast<double*>(scratch + mu_bytes);
    k_mu_to_working<T><<<(geo.K + 255) / 256, 256, 0, st>>>(mu, muT, geo.K);
    const dim3 grid((unsigned)((long long)chunks * batch));
    const size_t smem = 4 * (size_t)geo.chunk * sizeof(T);
    if (cplx)
        k_gcv_partials<T, true><<<grid, 256, smem, st>>>(reinterpret_cast<const C2<T>*>(ghat),
                                                          reinterpret_cast<const C2<T>*>(d), d_psf_stride, psf_per,
                                                          muT, geo, partials);
    else
        k_gcv_partials<T, false><<<grid, 256, smem, st>>>(reinterpret_cast<const T*>(ghat),
                                                           reinterpret_cast<const T*>(d), d_psf_stride, psf_per,
                                                           muT, geo, partials);
    cudaError_t e = launch_gcv_finalize_raw(partials, chunks, geo.K, batch, gcv, mu_idx, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error("hobc_gcv_noalloc launch", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

}  // namespace

extern "C" size_t hobc_gcv_noalloc_max_bytes(void) { return kScratchBytes; }

extern "C" hobc_status hobc_gcv_noalloc(const hobc_plan_desc* desc, const void* ghat_dev, const void* d_dev,
                                        const double* mu_dev, double* gcv_dev, int* mu_index_dev,
                                        void* cuda_stream) {
    if (!desc || !ghat_dev || !d_dev || !mu_dev || !mu_index_dev) return HOBC_ERR_ARG;
    const hobc_plan_desc& dsc = *desc;
    if (dsc.ndim != 1 && dsc.ndim != 2) return HOBC_ERR_ARG;
    if (dsc.n_mu < 1 || dsc.batch < 1) return HOBC_ERR_ARG;
    if (dsc.prec != HOBC_FP64 && dsc.prec != HOBC_FP32) return HOBC_ERR_ARG;
    if (dsc.L != HOBC_L_IDENTITY && dsc.L != HOBC_L_LAPLACIAN) return HOBC_ERR_ARG;
    if (dsc.psf_per_item != 0 && dsc.psf_per_item != 1) return HOBC_ERR_ARG;
    for (int i = 0; i < dsc.ndim; ++i)
        if (dsc.n[i] < 6 || dsc.n[i] > 1024) return HOBC_ERR_SIZE;
    int fam = dsc.family;
    if (fam == HOBC_FAMILY_AUTO) {
        if (dsc.bc_degree == 1) fam = dsc.psf_symmetric ? HOBC_FAMILY_SINE : -1;
        else if (dsc.bc_degree == 2) fam = dsc.psf_symmetric ? HOBC_FAMILY_COSINE : HOBC_FAMILY_FOURIER;
        else if (dsc.bc_degree == 3) fam = dsc.psf_symmetric ? HOBC_FAMILY_SINE_CUBIC : -1;
        else if (dsc.bc_degree == 4) fam = dsc.psf_symmetric ? HOBC_FAMILY_COSINE_QUARTIC : -1;
        else fam = -1;
        if (fam < 0) return HOBC_ERR_UNSUPPORTED;
    }
    if (fam != HOBC_FAMILY_COSINE_QUARTIC && (fam < HOBC_FAMILY_SINE || fam > HOBC_FAMILY_SINE_CUBIC))
        return HOBC_ERR_ARG;
    const bool two_borders = fam == HOBC_FAMILY_SINE_CUBIC || fam == HOBC_FAMILY_COSINE_QUARTIC;

    // geometry of the stored spectrum (include/hobc.h, "Spectrum layout")
    const int nl = dsc.n[dsc.ndim - 1];
    const int Nl = two_borders ? nl - 4 : nl - 2;
    const int Wl = fam == HOBC_FAMILY_FOURIER ? Nl / 2 + 3 : nl;
    const long long S = dsc.ndim == 1 ? (long long)Wl : (long long)Wl * dsc.n[0];
    const int chunk = hobc::gcv_chunk_for(S, dsc.n_mu, dsc.prec == HOBC_FP64);
    const long long chunks = (S + chunk - 1) / chunk;
    const size_t esz = dsc.prec == HOBC_FP64 ? 8 : 4;
    const size_t mu_bytes = ((size_t)dsc.n_mu * esz + 255) / 256 * 256;
    const double need = (double)mu_bytes + (double)dsc.batch * (double)chunks * 2.0 * dsc.n_mu * sizeof(double);
    if (need > (double)kScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "hobc_gcv_noalloc: needs %.0f bytes of scratch, the maximum is %zu "
                 "(batch x ceil(spectrum/chunk) x 2 x n_mu doubles plus the mu grid)",
                 need, kScratchBytes);
        hobc::set_last_error_text(msg);
        return HOBC_ERR_SIZE;
    }

    hobc::GcvGeom geo;
    geo.ndim = dsc.ndim;
    geo.fam = fam;
    geo.n0 = dsc.n[0];
    geo.N0 = two_borders ? dsc.n[0] - 4 : dsc.n[0] - 2;
    geo.n1 = nl;
    geo.N1 = Nl;
    geo.W1 = Wl;
    geo.lap = dsc.L == HOBC_L_LAPLACIAN;
    geo.S = S;
    geo.chunk = chunk;
    geo.K = dsc.n_mu;

    void* base = nullptr;
    hobc_status s = scratch_address(&base);
    if (s != HOBC_OK) return s;
    unsigned char* scratch = static_cast<unsigned char*>(base);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const int cplx = fam == HOBC_FAMILY_FOURIER;
    if (dsc.prec == HOBC_FP64)
        return launch<double>(geo, cplx, dsc.batch, (int)chunks, ghat_dev, d_dev, S, dsc.psf_per_item, mu_dev,
                              scratch, mu_bytes, gcv_dev, mu_index_dev, st);
    return launch<float>(geo, cplx, dsc.batch, (int)chunks, ghat_dev, d_dev, S, dsc.psf_per_item, mu_dev, scratch,
                         mu_bytes, gcv_dev, mu_index_dev, st);
}
