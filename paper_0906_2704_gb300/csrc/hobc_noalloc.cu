// hobc_gcv_noalloc: the GCV scan (per-CTA partial sums and the argmin) for
// callers that cannot allocate device memory.  The per-CTA partial sums -- the
// only scratch the scan needs -- and the FP32 copy of the mu grid live in one
// file-scope device array instead of a plan's cudaMalloc'd workspace.  The
// kernels are the ones hobc_gcv launches; only where their scratch lives differs.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include <cuda.h>

#include "hobc_internal.h"
#include "hobc_kernels.cuh"

namespace {

// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_gcv_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};               // device address of g_gcv_scratch, per device ...
unsigned long long g_scratch_ctx_id[kMaxDevices] = {};  // ... in the context with this unique id

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Driver entry points for the current context and its process-unique id, looked up once.
hobc_status driver_entry_points() {
    static cudaError_t lookup = cudaErrorUnknown;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        void* g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        lookup = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1);
        if (lookup == cudaSuccess)
            lookup = cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2);
        if (lookup == cudaSuccess &&
            (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f || !g))
            lookup = cudaErrorSymbolNotFound;
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(g);
    });
    if (lookup != cudaSuccess) {
        hobc::set_last_error("hobc_gcv_noalloc: driver entry points", lookup);
        return HOBC_ERR_CUDA;
    }
    return HOBC_OK;
}

// Unique id of the context current on this thread; false if none is current or
// it has been destroyed.
bool current_context_id(unsigned long long* id) {
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// the device current (cudaGetSymbolAddress, once per device) and kept.  The
// address belongs to the module loaded in the device's context; a device reset
// destroys that context and the next runtime call creates a new one in which the
// module has a new address.  So the address is kept together with the unique id
// of the context it was taken in, and looked up again when the current context
// has another id (or none yet: the lookup itself makes the runtime set it up).
hobc_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { hobc::set_last_error("hobc_gcv_noalloc: cudaGetDevice", e); return HOBC_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return HOBC_ERR_UNSUPPORTED;
    hobc_status s = driver_entry_points();
    if (s != HOBC_OK) return s;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    const bool have = current_context_id(&id);
    if (!have || !g_scratch_addr[dev] || id != g_scratch_ctx_id[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gcv_scratch);
        if (e != cudaSuccess) {
            hobc::set_last_error("hobc_gcv_noalloc: cudaGetSymbolAddress", e);
            return HOBC_ERR_CUDA;
        }
        if (!current_context_id(&id)) {
            hobc::set_last_error_text("hobc_gcv_noalloc: no current context after the symbol lookup");
            return HOBC_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
        g_scratch_ctx_id[dev] = id;
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
    if (geo.ndim == 1) {
        // as hobc_gcv does for 1D plans: one thread group per problem sums its whole
        // spectrum, so the scan needs no partial sums (only the grid in scratch)
        const int per = sizeof(T) == 4 ? 8 : 4;
        int tpi = 1;
        while (tpi * per < geo.K) tpi *= 2;
        if (tpi <= 32) {
            const unsigned grid = (unsigned)((batch + 256 / tpi - 1) / (256 / tpi));
#define HOBC_NOALLOC_ITEMS(TPI_)                                                                             \
    if (tpi == TPI_) {                                                                                       \
        if (cplx)                                                                                            \
            k_gcv_items<T, true, TPI_><<<grid, 256, 0, st>>>(reinterpret_cast<const C2<T>*>(ghat),          \
                                                             reinterpret_cast<const C2<T>*>(d), d_psf_stride, \
                                                             psf_per, muT, geo, batch, gcv, mu_idx);         \
        else                                                                                                 \
            k_gcv_items<T, false, TPI_><<<grid, 256, 0, st>>>(reinterpret_cast<const T*>(ghat),             \
                                                              reinterpret_cast<const T*>(d), d_psf_stride,   \
                                                              psf_per, muT, geo, batch, gcv, mu_idx);        \
    }
            HOBC_NOALLOC_ITEMS(1) HOBC_NOALLOC_ITEMS(2) HOBC_NOALLOC_ITEMS(4) HOBC_NOALLOC_ITEMS(8)
            HOBC_NOALLOC_ITEMS(16) HOBC_NOALLOC_ITEMS(32)
#undef HOBC_NOALLOC_ITEMS
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { set_last_error("hobc_gcv_noalloc launch", e); return HOBC_ERR_CUDA; }
            return HOBC_OK;
        }
    }
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
    // the same checks as hobc_plan_create (the PSF extents are not part of the request)
    int fam = 0;
    const hobc_status vs = hobc::resolve_desc(dsc, false, &fam);
    if (vs != HOBC_OK) return vs;
    if (dsc.prec != HOBC_FP64 && dsc.prec != HOBC_FP32) return HOBC_ERR_UNSUPPORTED;   // FFT-path spectra only
    // geometry of the stored spectrum (include/hobc.h, "Spectrum layout"): the
    // trigonometric order N of an axis and the stored entries of the last one
    const int nb = hobc::fam_nb(fam);
    auto order = [&](int n) { return fam == hobc::FAM_P ? n : n - 2 * nb; };
    const int nl = dsc.n[dsc.ndim - 1];
    const int Nl = order(nl);
    const int Wl = hobc::fam_fourier(fam) ? Nl / 2 + 1 + 2 * nb : nl;
    const long long S = dsc.ndim == 1 ? (long long)Wl : (long long)Wl * dsc.n[0];
    const int chunk = hobc::gcv_chunk_for(S, dsc.n_mu, dsc.prec == HOBC_FP64);
    const long long chunks = (S + chunk - 1) / chunk;
    const size_t esz = dsc.prec == HOBC_FP64 ? 8 : 4;
    const size_t mu_bytes = ((size_t)dsc.n_mu * esz + 255) / 256 * 256;
    // 1D problems run as hobc_gcv runs them (one thread group per problem, no
    // partial sums) when a group of at most 32 threads covers the grid
    int tpi = 1;
    while (tpi * (dsc.prec == HOBC_FP64 ? 4 : 8) < dsc.n_mu) tpi *= 2;
    const bool items_path = dsc.ndim == 1 && tpi <= 32;
    const double need = (double)mu_bytes +
                        (items_path ? 0.0 : (double)dsc.batch * (double)chunks * 2.0 * dsc.n_mu * sizeof(double));
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
    geo.N0 = order(dsc.n[0]);
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
    const int cplx = hobc::fam_fourier(fam);
    if (dsc.prec == HOBC_FP64)
        return launch<double>(geo, cplx, dsc.batch, (int)chunks, ghat_dev, d_dev, S, dsc.psf_per_item, mu_dev,
                              scratch, mu_bytes, gcv_dev, mu_index_dev, st);
    return launch<float>(geo, cplx, dsc.batch, (int)chunks, ghat_dev, d_dev, S, dsc.psf_per_item, mu_dev, scratch,
                         mu_bytes, gcv_dev, mu_index_dev, st);
}
