// C ABI of the method on 3D arrays (include/hobc_volume.h).  A volume plan
// wraps a 2D plan of its (n1, n2) slices (batch x n0 problems: tables of axes
// 1 and 2, the slice transforms, the mu grid) and adds the table of axis 0,
// the axis-0 workspace and the GCV partial sums; the launch sequences are in
// hobc_volume.cuh (instantiated per precision in hobc_f32.cu, hobc_f64.cu).
#include <algorithm>
#include <cstring>

#include "../../include/hobc_volume.h"
#include "hobc_internal.h"
#include "hobc_kernels.cuh"

using namespace hobc;

namespace {

void volume_free(hobc_volume_s* q) {
    if (!q) return;
    if (q->stream) cudaStreamSynchronize(q->stream);
    else cudaDeviceSynchronize();
    if (q->slice) hobc_plan_destroy(q->slice);
    free_axis(q->az);
    cudaFree(q->X); cudaFree(q->G); cudaFree(q->D); cudaFree(q->D2); cudaFree(q->partials); cudaFree(q->mu_idx);
    delete q;
}

template <typename T>
hobc_status dispatch_deblur(hobc_volume_s* q, const void* g, const void* psf, void* f, int* mi, double* gcv) {
    hobc_status s = run3_eig<T>(q, psf, q->D);
    if (s == HOBC_OK) s = run3_analysis<T>(q, g, q->G);
    if (s == HOBC_OK) s = run3_gcv<T>(q, q->G, q->D, gcv, mi);
    if (s == HOBC_OK) s = run3_synthesis<T>(q, q->G, f, q->D, mi);
    return s;
}

void begin(hobc_volume_s* q) { q->slice->launches = 0; }
void end(hobc_volume_s* q) { q->launches = q->slice->launches; }

}  // namespace

extern "C" {

hobc_status hobc_volume_create(const hobc_volume_desc* desc, const double* mu_grid_host, void* cuda_stream,
                               hobc_volume** out) {
    if (!out) return HOBC_ERR_ARG;
    *out = nullptr;
    if (!desc || !mu_grid_host) return HOBC_ERR_ARG;
    const hobc_volume_desc d = *desc;
    if (d.prec != HOBC_FP64 && d.prec != HOBC_FP32) return d.prec == HOBC_SPLIT_BF16 ? HOBC_ERR_UNSUPPORTED : HOBC_ERR_ARG;
    if (d.batch < 1 || d.n_mu < 1) return HOBC_ERR_ARG;
    if (d.n[0] < 6 || d.n[0] > 1024) return HOBC_ERR_SIZE;
    if (d.psf[0] < 1 || d.psf[0] % 2 == 0 || d.psf[0] > 63) return HOBC_ERR_SIZE;
    if ((long long)d.batch * d.n[0] > 65535) return HOBC_ERR_SIZE;      // slices ride on gridDim.y
    // the slice plan validates axes 1 and 2, the family, degree and symmetry
    hobc_plan_desc sd;
    memset(&sd, 0, sizeof(sd));
    sd.ndim = 2; sd.n[0] = d.n[1]; sd.n[1] = d.n[2]; sd.psf[0] = d.psf[1]; sd.psf[1] = d.psf[2];
    sd.bc_degree = d.bc_degree; sd.family = d.family; sd.psf_symmetric = d.psf_symmetric; sd.L = d.L;
    sd.prec = d.prec; sd.n_mu = d.n_mu; sd.batch = d.batch * d.n[0]; sd.psf_per_item = 0;
    hobc_volume_s* q = new hobc_volume_s();
    memset(q, 0, sizeof(*q));
    q->desc = d;
    q->prec = d.prec;
    q->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    q->K = d.n_mu;
    q->npsf = d.psf_per_item ? d.batch : 1;
    hobc_status s = hobc_plan_create(&sd, mu_grid_host, cuda_stream, &q->slice);
    if (s != HOBC_OK) { volume_free(q); return s; }
    q->fam = q->slice->fam;
    if (q->fam == HOBC_FAMILY_COSINE_QUARTIC || plain_only_family(q->fam)) {   // 2D and 1D only
        volume_free(q);
        return HOBC_ERR_UNSUPPORTED;
    }
    const int need = q->fam == HOBC_FAMILY_SINE_CUBIC ? 4 : 2;
    if (d.psf[0] > d.n[0] - need) { volume_free(q); return HOBC_ERR_SIZE; }
    const bool fp64 = d.prec == HOBC_FP64;
    cudaError_t e = fp64 ? build_axis_host<double>(q->az, q->fam, d.n[0], d.psf[0], false)
                         : build_axis_host<float>(q->az, q->fam, d.n[0], d.psf[0], false);
    q->S2 = q->slice->spec_elems;
    q->S3 = q->S2 * (size_t)d.n[0];
    q->esz = (q->fam == HOBC_FAMILY_FOURIER ? 2 : 1) * (fp64 ? sizeof(double) : sizeof(float));
    q->chunk = gcv_chunk_for((long long)q->S3, q->K, fp64);
    q->chunks = (int)(((long long)q->S3 + q->chunk - 1) / q->chunk);
    const size_t B = (size_t)d.batch;
    auto alloc = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    alloc(&q->X, B * q->S3 * q->esz);
    alloc(&q->G, B * q->S3 * q->esz);
    alloc(&q->D, (size_t)q->npsf * q->S3 * q->esz);
    alloc(&q->D2, (size_t)q->npsf * d.psf[0] * q->S2 * q->esz);
    alloc((void**)&q->partials, B * q->chunks * 2 * (size_t)q->K * sizeof(double));
    alloc((void**)&q->mu_idx, B * sizeof(int));
    if (e != cudaSuccess) {
        set_last_error("hobc_volume_create", e);
        volume_free(q);
        return HOBC_ERR_CUDA;
    }
    *out = q;
    return HOBC_OK;
}

void hobc_volume_destroy(hobc_volume* q) { volume_free(q); }

hobc_status hobc_volume_spectrum_size(const hobc_volume* q, size_t* spec, int* cplx) {
    if (!q || !spec || !cplx) return HOBC_ERR_ARG;
    *spec = q->S3;
    *cplx = q->fam == HOBC_FAMILY_FOURIER;
    return HOBC_OK;
}

hobc_status hobc_volume_analysis(hobc_volume* q, const void* g, void* ghat) {
    if (!q || !g || !ghat) return HOBC_ERR_ARG;
    begin(q);
    hobc_status s = q->prec == HOBC_FP64 ? run3_analysis<double>(q, g, ghat) : run3_analysis<float>(q, g, ghat);
    end(q);
    return s;
}

hobc_status hobc_volume_synthesis(hobc_volume* q, const void* c, void* y) {
    if (!q || !c || !y) return HOBC_ERR_ARG;
    begin(q);
    hobc_status s = q->prec == HOBC_FP64 ? run3_synthesis<double>(q, c, y, nullptr, nullptr)
                                         : run3_synthesis<float>(q, c, y, nullptr, nullptr);
    end(q);
    return s;
}

hobc_status hobc_volume_eigenvalues(hobc_volume* q, const void* psf, void* d) {
    if (!q || !psf || !d) return HOBC_ERR_ARG;
    begin(q);
    hobc_status s = q->prec == HOBC_FP64 ? run3_eig<double>(q, psf, d) : run3_eig<float>(q, psf, d);
    end(q);
    return s;
}

hobc_status hobc_volume_gcv(hobc_volume* q, const void* ghat, const void* d, double* gcv, int* mu_idx) {
    if (!q || !ghat || !d || !mu_idx) return HOBC_ERR_ARG;
    begin(q);
    hobc_status s = q->prec == HOBC_FP64 ? run3_gcv<double>(q, ghat, d, gcv, mu_idx)
                                         : run3_gcv<float>(q, ghat, d, gcv, mu_idx);
    end(q);
    return s;
}

hobc_status hobc_volume_filter_synthesis(hobc_volume* q, const void* ghat, const void* d, const int* mu_idx, void* f) {
    if (!q || !ghat || !d || !mu_idx || !f) return HOBC_ERR_ARG;
    begin(q);
    hobc_status s = q->prec == HOBC_FP64 ? run3_synthesis<double>(q, ghat, f, d, mu_idx)
                                         : run3_synthesis<float>(q, ghat, f, d, mu_idx);
    end(q);
    return s;
}

hobc_status hobc_volume_deblur(hobc_volume* q, const void* g, const void* psf, void* f, int* mu_idx, double* gcv) {
    if (!q || !g || !psf || !f) return HOBC_ERR_ARG;
    if (g == f) return HOBC_ERR_ARG;
    int* mi = mu_idx ? mu_idx : q->mu_idx;
    begin(q);
    hobc_status s = q->prec == HOBC_FP64 ? dispatch_deblur<double>(q, g, psf, f, mi, gcv)
                                         : dispatch_deblur<float>(q, g, psf, f, mi, gcv);
    end(q);
    return s;
}

int hobc_volume_launch_count(const hobc_volume* q) { return q ? q->launches : 0; }

}  // extern "C"
