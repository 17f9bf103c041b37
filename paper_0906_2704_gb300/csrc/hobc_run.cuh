// Launch sequences of the hot path, templated on the working precision.
// Included once per precision (hobc_f32.cu, hobc_f64.cu).
#pragma once

#include <algorithm>

#include "hobc_internal.h"
#include "hobc_kernels.cuh"

namespace hobc {

template <typename T>
static Axis<T> dev_axis(const AxisHost& a) {
    Axis<T> x;
    x.fam = a.fam; x.n = a.n; x.N = a.N; x.L = a.L; x.M = a.M; x.log2M = a.log2M;
    x.blue = a.blue; x.tpg = a.tpg; x.r16 = a.r16; x.Mp = group_slots(a.M); x.H = a.H; x.W = a.W;
    x.sslot = a.sslot;
    x.tw = reinterpret_cast<const C2<T>*>(a.tw);
    x.chirp = reinterpret_cast<const C2<T>*>(a.chirp);
    x.bhat = reinterpret_cast<const C2<T>*>(a.bhat);
    x.post = reinterpret_cast<const C2<T>*>(a.post);
    x.q = reinterpret_cast<const T*>(a.q);
    x.q2 = reinterpret_cast<const T*>(a.q2);
    x.ka = a.ka; x.kb = a.kb;
    for (int i = 0; i < 16; ++i) x.k4[i] = a.k4[i];
    x.q1 = (T)a.q1; x.sc = (T)a.sc; x.s0 = (T)a.s0; x.s1 = (T)a.s1;
    x.is0 = (T)a.is0; x.is1 = (T)a.is1; x.invN = (T)a.invN;
    return x;
}

// Groups per CTA for a kernel working on pairs of real lines (stage = 2G lines
// of W entries of `ebytes`); a transposed store wants 2G * ebytes >= 32 bytes.
static inline Launch pair_launch(const AxisHost& a, size_t cbytes, size_t ebytes, int nlines, int items,
                                 bool transposed) {
    int G = std::max(1, 256 / a.tpg);
    if (transposed) G = std::max(G, (int)((32 + 2 * ebytes - 1) / (2 * ebytes)));
    G = std::min(G, std::max(1, 512 / a.tpg));
    G = std::min(G, (nlines + 1) / 2);
    G = std::max(G, 1);
    const size_t Mp = (size_t)group_slots(a.M);
    auto smem = [&](int g) { return (size_t)g * Mp * cbytes + (a.sslot >= 0 ? 0 : (size_t)2 * g * a.W * ebytes); };
    while (G > 1 && smem(G) > 200 * 1024) --G;
    Launch l;
    l.block = dim3(G * a.tpg);
    l.grid = dim3((nlines + 2 * G - 1) / (2 * G), items);
    l.smem = smem(G);
    return l;
}

static inline Launch cplx_launch(const AxisHost& a, size_t cbytes, int nlines, int items) {
    int G = std::max(1, 256 / a.tpg);
    G = std::min(G, std::max(1, 512 / a.tpg));
    G = std::min(G, nlines);
    const size_t Mp = (size_t)group_slots(a.M);
    while (G > 1 && (size_t)G * Mp * cbytes > 200 * 1024) --G;
    Launch l;
    l.block = dim3(G * a.tpg);
    l.grid = dim3((nlines + G - 1) / G, items);
    l.smem = (size_t)G * Mp * cbytes;
    return l;
}

static inline hobc_status check_launch(hobc_plan_s* p, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(what, e);
        return HOBC_ERR_CUDA;
    }
    ++p->launches;
    return HOBC_OK;
}

template <typename T, int FAM>
static hobc_status pair_analysis(hobc_plan_s* p, const AxisHost& a, const T* in, long long in_item,
                                 long long in_rs, void* out, long long out_item, long long out_rs,
                                 long long out_cs, int nlines, int items) {
    typedef typename ElemT<T, fam_fourier(FAM)>::t E;
    Launch l = pair_launch(a, sizeof(C2<T>), sizeof(E), nlines, items, out_rs == 1);
    k_pair_analysis<T, FAM><<<l.grid, l.block, l.smem, p->stream>>>(
        in, in_item, in_rs, reinterpret_cast<E*>(out), out_item, out_rs, out_cs, nlines, dev_axis<T>(a));
    return check_launch(p, "k_pair_analysis");
}

template <typename T, int FAM, int FMODE>
static hobc_status pair_synthesis(hobc_plan_s* p, const AxisHost& a, const void* in, long long in_item,
                                  long long in_rs, long long in_cs, T* out, long long out_item,
                                  long long out_rs, int nlines, int items, const FilterDesc& fd) {
    typedef typename ElemT<T, fam_fourier(FAM)>::t E;
    Launch l = pair_launch(a, sizeof(C2<T>), sizeof(E), nlines, items, in_rs == 1);
    k_pair_synthesis<T, FAM, FMODE><<<l.grid, l.block, l.smem, p->stream>>>(
        reinterpret_cast<const E*>(in), in_item, in_rs, in_cs, out, out_item, out_rs, nlines, dev_axis<T>(a), fd);
    return check_launch(p, "k_pair_synthesis");
}

static inline FilterDesc make_filter(const hobc_plan_s* p, const void* D, const int* mu_idx) {
    FilterDesc f;
    f.D = D;
    f.d_psf_stride = (long long)p->spec_elems;
    f.psf_per = p->desc.psf_per_item;
    f.mu_idx = mu_idx;
    f.mu = p->mu;
    f.K = p->K;
    f.lap = p->desc.L == HOBC_L_LAPLACIAN;
    const AxisHost& o = p->ax[p->nax - 1];
    f.o_fam = o.fam; f.o_n = o.n; f.o_N = o.N; f.o_W = o.W;
    f.mu_val = nullptr;
    return f;
}

// -------------------------------------------------------------- analysis

template <typename T, int FAM>
static hobc_status analysis_fam(hobc_plan_s* p, const T* g, void* ghat) {
    const int B = p->desc.batch;
    if (p->nax == 1) {
        const AxisHost& a = p->ax[0];
        return pair_analysis<T, FAM>(p, a, g, 0, a.n, ghat, 0, a.W, 1, B, 1);
    }
    const AxisHost& a0 = p->ax[0];
    const AxisHost& a1 = p->ax[1];
    const long long S = (long long)p->spec_elems;
    const int n0 = a0.n, n1 = a1.n;
    hobc_status s = pair_analysis<T, FAM>(p, a1, g, (long long)n0 * n1, n1, p->R, S, 1, n0, n0, B);
    if (s != HOBC_OK) return s;
    if constexpr (fam_fourier(FAM)) {
        Launch l = cplx_launch(a0, sizeof(C2<T>), a1.W, B);
        k_cplx_analysis<T, FAM><<<l.grid, l.block, l.smem, p->stream>>>(
            reinterpret_cast<const C2<T>*>(p->R), reinterpret_cast<C2<T>*>(ghat), S, a1.W, dev_axis<T>(a0));
        return check_launch(p, "k_cplx_analysis");
    } else {
        return pair_analysis<T, FAM>(p, a0, reinterpret_cast<const T*>(p->R), S, n0, ghat, S, n0, 1, n1, B);
    }
}

template <typename T>
hobc_status run_analysis(hobc_plan_s* p, const void* g, void* ghat) {
    if (sizeof(T) == 4 && p->prec == HOBC_SPLIT_BF16) return dense_analysis(p, g, ghat);
    const T* gt = reinterpret_cast<const T*>(g);
    switch (p->fam) {
        case FAM_S: return analysis_fam<T, FAM_S>(p, gt, ghat);
        case FAM_S3: return analysis_fam<T, FAM_S3>(p, gt, ghat);
        case FAM_C4: return analysis_fam<T, FAM_C4>(p, gt, ghat);
        case FAM_C: return analysis_fam<T, FAM_C>(p, gt, ghat);
        case FAM_P: return analysis_fam<T, FAM_P>(p, gt, ghat);
        case FAM_F4:
            if constexpr (sizeof(T) == 8) return analysis_fam<T, FAM_F4>(p, gt, ghat);   // FP64 only
            return HOBC_ERR_UNSUPPORTED;
        default: return analysis_fam<T, FAM_F>(p, gt, ghat);
    }
}

// ------------------------------------------------------------- synthesis

template <typename T, int FAM, bool FILTER>
static hobc_status synthesis_fam(hobc_plan_s* p, const void* c, T* y, const FilterDesc& fd) {
    const int B = p->desc.batch;
    if (p->nax == 1) {
        const AxisHost& a = p->ax[0];
        return pair_synthesis<T, FAM, FILTER ? 1 : 0>(p, a, c, 0, a.W, 1, y, 0, a.n, B, 1, fd);
    }
    const AxisHost& a0 = p->ax[0];
    const AxisHost& a1 = p->ax[1];
    const long long S = (long long)p->spec_elems;
    const int n0 = a0.n, n1 = a1.n;
    hobc_status s;
    if constexpr (fam_fourier(FAM)) {
        Launch l = cplx_launch(a0, sizeof(C2<T>), a1.W, B);
        k_cplx_synthesis<T, FAM, FILTER><<<l.grid, l.block, l.smem, p->stream>>>(
            reinterpret_cast<const C2<T>*>(c), reinterpret_cast<C2<T>*>(p->R), S, a1.W, dev_axis<T>(a0), fd);
        s = check_launch(p, "k_cplx_synthesis");
    } else {
        s = pair_synthesis<T, FAM, FILTER ? 2 : 0>(p, a0, c, S, n0, 1, reinterpret_cast<T*>(p->R), S, n0, n1, B, fd);
    }
    if (s != HOBC_OK) return s;
    FilterDesc none = fd;
    return pair_synthesis<T, FAM, 0>(p, a1, p->R, S, 1, n0, y, (long long)n0 * n1, n1, n0, B, none);
}

template <typename T>
hobc_status run_synthesis(hobc_plan_s* p, const void* c, void* y) {
    if (sizeof(T) == 4 && p->prec == HOBC_SPLIT_BF16) return dense_synthesis(p, c, y);
    FilterDesc fd = make_filter(p, nullptr, nullptr);
    T* yt = reinterpret_cast<T*>(y);
    switch (p->fam) {
        case FAM_S: return synthesis_fam<T, FAM_S, false>(p, c, yt, fd);
        case FAM_S3: return synthesis_fam<T, FAM_S3, false>(p, c, yt, fd);
        case FAM_C4: return synthesis_fam<T, FAM_C4, false>(p, c, yt, fd);
        case FAM_C: return synthesis_fam<T, FAM_C, false>(p, c, yt, fd);
        case FAM_P: return synthesis_fam<T, FAM_P, false>(p, c, yt, fd);
        case FAM_F4:
            if constexpr (sizeof(T) == 8) return synthesis_fam<T, FAM_F4, false>(p, c, yt, fd);
            return HOBC_ERR_UNSUPPORTED;
        default: return synthesis_fam<T, FAM_F, false>(p, c, yt, fd);
    }
}

template <typename T>
hobc_status run_filter_synthesis(hobc_plan_s* p, const void* ghat, const void* D, const int* mu_idx, void* f) {
    if (sizeof(T) == 4 && p->prec == HOBC_SPLIT_BF16) return dense_filter_synthesis(p, ghat, D, mu_idx, nullptr, f);
    FilterDesc fd = make_filter(p, D, mu_idx);
    T* ft = reinterpret_cast<T*>(f);
    switch (p->fam) {
        case FAM_S: return synthesis_fam<T, FAM_S, true>(p, ghat, ft, fd);
        case FAM_S3: return synthesis_fam<T, FAM_S3, true>(p, ghat, ft, fd);
        case FAM_C4: return synthesis_fam<T, FAM_C4, true>(p, ghat, ft, fd);
        case FAM_C: return synthesis_fam<T, FAM_C, true>(p, ghat, ft, fd);
        case FAM_P: return synthesis_fam<T, FAM_P, true>(p, ghat, ft, fd);
        case FAM_F4:
            if constexpr (sizeof(T) == 8) return synthesis_fam<T, FAM_F4, true>(p, ghat, ft, fd);
            return HOBC_ERR_UNSUPPORTED;
        default: return synthesis_fam<T, FAM_F, true>(p, ghat, ft, fd);
    }
}

// The same with mu* given per problem as a value rather than a grid index.
template <typename T>
hobc_status run_filter_synthesis_mu(hobc_plan_s* p, const void* ghat, const void* D, const double* mu_val, void* f) {
    if (sizeof(T) == 4 && p->prec == HOBC_SPLIT_BF16) return dense_filter_synthesis(p, ghat, D, nullptr, mu_val, f);
    FilterDesc fd = make_filter(p, D, nullptr);
    fd.mu_val = mu_val;
    T* ft = reinterpret_cast<T*>(f);
    switch (p->fam) {
        case FAM_S: return synthesis_fam<T, FAM_S, true>(p, ghat, ft, fd);
        case FAM_S3: return synthesis_fam<T, FAM_S3, true>(p, ghat, ft, fd);
        case FAM_C4: return synthesis_fam<T, FAM_C4, true>(p, ghat, ft, fd);
        case FAM_C: return synthesis_fam<T, FAM_C, true>(p, ghat, ft, fd);
        case FAM_P: return synthesis_fam<T, FAM_P, true>(p, ghat, ft, fd);
        case FAM_F4:
            if constexpr (sizeof(T) == 8) return synthesis_fam<T, FAM_F4, true>(p, ghat, ft, fd);
            return HOBC_ERR_UNSUPPORTED;
        default: return synthesis_fam<T, FAM_F, true>(p, ghat, ft, fd);
    }
}

// ----------------------------------------------------------- eigenvalues

template <typename T>
hobc_status run_eig(hobc_plan_s* p, const void* psf, void* D) {
    const AxisHost& last = p->ax[p->nax - 1];
    const bool cplx = fam_fourier(p->fam);
    const double2* E0;
    const float4* E0f;
    int p0, n0;
    if (p->nax == 2) { E0 = p->ax[0].etab; E0f = p->ax[0].etab2; p0 = p->ax[0].p; n0 = p->ax[0].n; }
    else {                                              // unit entry after the table
        E0 = last.etab + (size_t)last.W * last.p;
        E0f = last.etab2 + (size_t)last.W * last.p;
        p0 = 1;
        n0 = 1;
    }
    const long long psf_stride = (long long)p->psf_elems;
    dim3 grid(p->npsf, last.W);
    if (cplx)
        k_eig<T, true><<<grid, 256, 0, p->stream>>>(reinterpret_cast<const T*>(psf), psf_stride, p0, last.p, E0,
                                                    last.etab, E0f, n0, reinterpret_cast<C2<T>*>(D),
                                                    (long long)p->spec_elems);
    else
        k_eig<T, false><<<grid, 256, 0, p->stream>>>(reinterpret_cast<const T*>(psf), psf_stride, p0, last.p, E0,
                                                     last.etab, E0f, n0, reinterpret_cast<T*>(D),
                                                     (long long)p->spec_elems);
    return check_launch(p, "k_eig");
}

// ------------------------------------------------------------------ GCV

template <typename T>
hobc_status run_gcv(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    if constexpr (sizeof(T) == 4)
        if (gcvx_active(p) && p->nax == 2) return run_gcv_expansion(p, ghat, D, gcv, mu_idx);
    GcvGeom geo;
    const AxisHost& last = p->ax[p->nax - 1];
    geo.ndim = p->nax;
    geo.fam = p->fam;
    geo.n0 = p->ax[0].n;
    geo.N0 = p->ax[0].N;
    geo.n1 = last.n;
    geo.N1 = last.N;
    geo.W1 = last.W;
    geo.lap = p->desc.L == HOBC_L_LAPLACIAN;
    geo.S = (long long)p->spec_elems;
    geo.chunk = p->gcv_chunk;
    geo.K = p->K;
    if (p->nax == 1) {
        // many small spectra: one thread group per problem, no partial sums
        const int per = sizeof(T) == 4 ? 8 : 4;
        int tpi = 1;
        while (tpi * per < p->K) tpi *= 2;
        if (tpi <= 32) {
            const int B = p->desc.batch;
            const unsigned grid = (unsigned)((B + 256 / tpi - 1) / (256 / tpi));
            typedef typename ElemT<T, true>::t CT;
#define HOBC_ITEMS(TPI_)                                                                                   \
    if (tpi == TPI_) {                                                                                     \
        if (fam_fourier(p->fam))                                                                           \
            k_gcv_items<T, true, TPI_><<<grid, 256, 0, p->stream>>>(                                        \
                reinterpret_cast<const CT*>(ghat), reinterpret_cast<const CT*>(D), (long long)p->spec_elems, \
                p->desc.psf_per_item, reinterpret_cast<const T*>(p->muT), geo, B, gcv, mu_idx);            \
        else                                                                                               \
            k_gcv_items<T, false, TPI_><<<grid, 256, 0, p->stream>>>(                                       \
                reinterpret_cast<const T*>(ghat), reinterpret_cast<const T*>(D), (long long)p->spec_elems,  \
                p->desc.psf_per_item, reinterpret_cast<const T*>(p->muT), geo, B, gcv, mu_idx);            \
    }
            HOBC_ITEMS(1) HOBC_ITEMS(2) HOBC_ITEMS(4) HOBC_ITEMS(8) HOBC_ITEMS(16) HOBC_ITEMS(32)
#undef HOBC_ITEMS
            return check_launch(p, "k_gcv_items");
        }
    }
    dim3 grid((unsigned)(p->gcv_chunks * (long long)p->desc.batch));
    const size_t smem = 4 * (size_t)p->gcv_chunk * sizeof(T);
    if (fam_fourier(p->fam))
        k_gcv_partials<T, true><<<grid, 256, smem, p->stream>>>(
            reinterpret_cast<const C2<T>*>(ghat), reinterpret_cast<const C2<T>*>(D), (long long)p->spec_elems,
            p->desc.psf_per_item, reinterpret_cast<const T*>(p->muT), geo, p->partials);
    else
        k_gcv_partials<T, false><<<grid, 256, smem, p->stream>>>(
            reinterpret_cast<const T*>(ghat), reinterpret_cast<const T*>(D), (long long)p->spec_elems,
            p->desc.psf_per_item, reinterpret_cast<const T*>(p->muT), geo, p->partials);
    hobc_status s = check_launch(p, "k_gcv_partials");
    if (s != HOBC_OK) return s;
    return launch_gcv_finalize(p, gcv, mu_idx);
}

// Shared-memory share of the unified L1/shared array requested for the line
// kernels (percent; -1 leaves the choice to the driver, which keeps enough L1
// for the twiddle, chirp and border tables: 4% faster than 100 at 1024^2).
#ifndef HOBC_CARVEOUT
#define HOBC_CARVEOUT -1
#endif

// Allow the line kernels up to 200 KB of dynamic shared memory.
template <typename T>
hobc_status prepare_kernels(hobc_plan_s* p) {
    const int lim = 200 * 1024;
    cudaError_t e = cudaSuccess;
#define HOBC_SMEM(k)                                                                                \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, HOBC_CARVEOUT)
    HOBC_SMEM((k_pair_analysis<T, FAM_S>));
    HOBC_SMEM((k_pair_analysis<T, FAM_S3>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_S3, 0>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_S3, 1>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_S3, 2>));
    HOBC_SMEM((k_pair_analysis<T, FAM_C4>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_C4, 0>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_C4, 1>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_C4, 2>));
    HOBC_SMEM((k_pair_analysis<T, FAM_C>));
    HOBC_SMEM((k_pair_analysis<T, FAM_F>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_S, 0>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_S, 1>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_S, 2>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_C, 0>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_C, 1>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_C, 2>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_F, 0>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_F, 1>));
    HOBC_SMEM((k_cplx_analysis<T, FAM_F>));
    HOBC_SMEM((k_cplx_synthesis<T, FAM_F, false>));
    HOBC_SMEM((k_cplx_synthesis<T, FAM_F, true>));
    HOBC_SMEM((k_pair_analysis<T, FAM_P>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_P, 0>));
    HOBC_SMEM((k_pair_synthesis<T, FAM_P, 1>));
    HOBC_SMEM((k_cplx_analysis<T, FAM_P>));
    HOBC_SMEM((k_cplx_synthesis<T, FAM_P, false>));
    HOBC_SMEM((k_cplx_synthesis<T, FAM_P, true>));
    if constexpr (sizeof(T) == 8) {
        HOBC_SMEM((k_pair_analysis<T, FAM_F4>));
        HOBC_SMEM((k_pair_synthesis<T, FAM_F4, 0>));
        HOBC_SMEM((k_pair_synthesis<T, FAM_F4, 1>));
        HOBC_SMEM((k_cplx_analysis<T, FAM_F4>));
        HOBC_SMEM((k_cplx_synthesis<T, FAM_F4, false>));
        HOBC_SMEM((k_cplx_synthesis<T, FAM_F4, true>));
    }
    HOBC_SMEM((k_gcv_partials<T, false>));
    HOBC_SMEM((k_gcv_partials<T, true>));
#undef HOBC_SMEM
    if (e != cudaSuccess) {
        set_last_error("cudaFuncSetAttribute", e);
        return HOBC_ERR_CUDA;
    }
    return HOBC_OK;
}

}  // namespace hobc

#include "hobc_volume.cuh"

#define HOBC_INSTANTIATE(T)                                                                                  \
    template hobc_status hobc::run_eig<T>(hobc_plan_s*, const void*, void*);                                 \
    template hobc_status hobc::run_analysis<T>(hobc_plan_s*, const void*, void*);                            \
    template hobc_status hobc::run_synthesis<T>(hobc_plan_s*, const void*, void*);                           \
    template hobc_status hobc::run_gcv<T>(hobc_plan_s*, const void*, const void*, double*, int*);            \
    template hobc_status hobc::run_filter_synthesis<T>(hobc_plan_s*, const void*, const void*, const int*,   \
                                                       void*);                                               \
    template hobc_status hobc::run_filter_synthesis_mu<T>(hobc_plan_s*, const void*, const void*,             \
                                                          const double*, void*);                             \
    template hobc_status hobc::prepare_kernels<T>(hobc_plan_s*);                                             \
    template hobc_status hobc::run3_analysis<T>(hobc_volume_s*, const void*, void*);                         \
    template hobc_status hobc::run3_synthesis<T>(hobc_volume_s*, const void*, void*, const void*, const int*); \
    template hobc_status hobc::run3_eig<T>(hobc_volume_s*, const void*, void*);                              \
    template hobc_status hobc::run3_gcv<T>(hobc_volume_s*, const void*, const void*, double*, int*);
