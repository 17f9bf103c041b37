// Launch sequences of the method on 3D arrays (Sec. 6; include/hobc_volume.h),
// templated on the working precision; included by hobc_run.cuh after the 2D
// sequences it builds on.  Analysis: the 2D analysis of every (n1, n2) slice
// ([batch][n0][S2]), a transpose to [batch][S2][n0], and the line transform
// along axis 0 (real lines for the real families, complex lines for the
// Fourier family).  Synthesis runs the same steps backwards; the filter at mu*
// is a separate pass over the volume spectrum.
#pragma once

namespace hobc {

// [b][R][C] -> [b][C][R] through a 32 x 33 shared tile.
// grid = (ceil(C / 32), ceil(R / 32), batch), block = (32, 8).
template <typename E>
__global__ void __launch_bounds__(256)
k_vol_transpose(const E* __restrict__ in, E* __restrict__ out, int R, long long C) {
    __shared__ E tile[32][33];
    const long long b = blockIdx.z;
    const E* src = in + b * (long long)R * C;
    E* dst = out + b * (long long)R * C;
    const long long c0 = (long long)blockIdx.x * 32;
    const int r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k;
        const long long c = c0 + threadIdx.x;
        if (r < R && c < C) tile[k][threadIdx.x] = src[(long long)r * C + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const long long c = c0 + k;
        const int r = r0 + threadIdx.x;
        if (r < R && c < C) dst[c * R + r] = tile[threadIdx.x][k];
    }
}

// 3D eigenvalues from those of the PSF's slices: the 3D symbol at
// (-theta_t0, -theta_t1, -theta_t2) is sum_j0 exp(-i (j0 - m0) theta_t0)
// d2_j0(t1, t2), with d2_j0 the 2D eigenvalues of slice j0 (FP64 sums; real
// families keep the real part, the imaginary one cancels for a PSF symmetric
// along axis 0).  One CTA per slice entry e2 (its p0 slice values staged in
// shared memory), threads over t0, so each CTA writes nz consecutive entries.
// grid = (S2, PSFs), block = min(nz, 256) rounded to a warp.
template <typename T, bool CPLX>
__global__ void __launch_bounds__(256)
k_vol_eig(const typename ElemT<T, CPLX>::t* __restrict__ D2, int p0, long long S2, const double2* __restrict__ Ez,
          int nz, typename ElemT<T, CPLX>::t* __restrict__ D3, long long S3) {
    typedef typename ElemT<T, CPLX>::t E;
    __shared__ double2 v[64];
    const long long e2 = blockIdx.x;
    const long long ip = blockIdx.y;
    for (int j = threadIdx.x; j < p0; j += blockDim.x) {
        const E d = D2[(ip * p0 + j) * S2 + e2];
        if constexpr (CPLX) v[j] = make_double2((double)d.x, (double)d.y);
        else v[j] = make_double2((double)d, 0.0);
    }
    __syncthreads();
    E* o = D3 + ip * S3 + e2 * nz;
    for (int tz = threadIdx.x; tz < nz; tz += blockDim.x) {
        double re = 0, im = 0;
        for (int j = 0; j < p0; ++j) {
            const double2 e = Ez[(long long)tz * p0 + j];
            re += e.x * v[j].x - e.y * v[j].y;
            im += e.x * v[j].y + e.y * v[j].x;
        }
        if constexpr (CPLX) o[tz] = cmk<T>((T)re, (T)im);
        else o[tz] = (T)re;
    }
}

// conj(d) ghat / (|d|^2 + mu* |s|^2) on every entry of the volume spectrum
// (Eq. (eq:freg)), mu* = grid[mu_idx[item]] (clamped to the grid).
// grid = (ceil(S3 / 256), items), block = 256.
template <typename T, bool CPLX>
__global__ void k_vol_filter(const typename ElemT<T, CPLX>::t* __restrict__ gh,
                             const typename ElemT<T, CPLX>::t* __restrict__ D, int psf_per, GcvGeom geo,
                             const int* __restrict__ mu_idx, const double* __restrict__ mu, int K,
                             typename ElemT<T, CPLX>::t* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= geo.S) return;
    const long long item = blockIdx.y;
    const int k = min(max(mu_idx[item], 0), K - 1);
    int c;
    const T s2 = lap_s2<T>(geo, e, c);
    out[item * geo.S + e] = apply_filter(gh[item * geo.S + e], D[(psf_per ? item : 0) * geo.S + e], s2, (T)mu[k]);
}

template <typename T>
static GcvGeom vol_geo(const hobc_volume_s* q) {
    GcvGeom geo;
    memset(&geo, 0, sizeof(geo));
    const hobc_plan_s* sl = q->slice;
    geo.ndim = 3;
    geo.fam = q->fam;
    geo.n0 = sl->ax[0].n; geo.N0 = sl->ax[0].N;
    geo.n1 = sl->ax[1].n; geo.N1 = sl->ax[1].N; geo.W1 = sl->ax[1].W;
    geo.nz = q->az.n; geo.Nz = q->az.N;
    geo.lap = q->desc.L == HOBC_L_LAPLACIAN;
    geo.S = (long long)q->S3;
    geo.chunk = q->chunk;
    geo.K = q->K;
    return geo;
}

template <typename E>
static hobc_status vol_transpose(hobc_volume_s* q, const void* in, void* out, int R, long long C) {
    const dim3 grid((unsigned)((C + 31) / 32), (unsigned)((R + 31) / 32), (unsigned)q->desc.batch);
    k_vol_transpose<E><<<grid, dim3(32, 8), 0, q->stream>>>(reinterpret_cast<const E*>(in), reinterpret_cast<E*>(out),
                                                            R, C);
    return check_launch(q->slice, "k_vol_transpose");
}

template <typename T>
hobc_status run3_analysis(hobc_volume_s* q, const void* g, void* ghat) {
    hobc_plan_s* sl = q->slice;
    const int B = q->desc.batch, n0 = q->desc.n[0];
    const long long S2 = (long long)q->S2, S3 = (long long)q->S3;
    hobc_status s = run_analysis<T>(sl, g, sl->G);                 // [B][n0][S2]
    if (s != HOBC_OK) return s;
    if (q->fam == FAM_F) {
        s = vol_transpose<C2<T>>(q, sl->G, q->X, n0, S2);           // [B][S2][n0]
        if (s != HOBC_OK) return s;
        Launch l = cplx_launch(q->az, sizeof(C2<T>), (int)S2, B);
        k_cplx_analysis<T, FAM_F><<<l.grid, l.block, l.smem, q->stream>>>(reinterpret_cast<const C2<T>*>(q->X),
                                                                   reinterpret_cast<C2<T>*>(ghat), S3, (int)S2,
                                                                   dev_axis<T>(q->az));
        return check_launch(sl, "k_cplx_analysis");
    }
    s = vol_transpose<T>(q, sl->G, q->X, n0, S2);
    if (s != HOBC_OK) return s;
    const T* x = reinterpret_cast<const T*>(q->X);
    switch (q->fam) {
        case FAM_S: return pair_analysis<T, FAM_S>(sl, q->az, x, S3, n0, ghat, S3, n0, 1, (int)S2, B);
        case FAM_S3: return pair_analysis<T, FAM_S3>(sl, q->az, x, S3, n0, ghat, S3, n0, 1, (int)S2, B);
        default: return pair_analysis<T, FAM_C>(sl, q->az, x, S3, n0, ghat, S3, n0, 1, (int)S2, B);
    }
}

template <typename T>
hobc_status run3_synthesis(hobc_volume_s* q, const void* c, void* y, const void* D, const int* mu_idx) {
    hobc_plan_s* sl = q->slice;
    const int B = q->desc.batch, n0 = q->desc.n[0];
    const long long S2 = (long long)q->S2, S3 = (long long)q->S3;
    const bool F = q->fam == FAM_F;
    const void* src = c;
    hobc_status s = HOBC_OK;
    if (D) {                                                        // filter into the slice plan's workspace
        const GcvGeom geo = vol_geo<T>(q);
        const dim3 grid((unsigned)((S3 + 255) / 256), (unsigned)B);
        if (F)
            k_vol_filter<T, true><<<grid, 256, 0, q->stream>>>(reinterpret_cast<const C2<T>*>(c),
                                                               reinterpret_cast<const C2<T>*>(D), q->desc.psf_per_item,
                                                               geo, mu_idx, sl->mu, q->K,
                                                               reinterpret_cast<C2<T>*>(sl->G));
        else
            k_vol_filter<T, false><<<grid, 256, 0, q->stream>>>(reinterpret_cast<const T*>(c),
                                                                reinterpret_cast<const T*>(D), q->desc.psf_per_item,
                                                                geo, mu_idx, sl->mu, q->K, reinterpret_cast<T*>(sl->G));
        s = check_launch(sl, "k_vol_filter");
        if (s != HOBC_OK) return s;
        src = sl->G;
    }
    FilterDesc none = make_filter(sl, nullptr, nullptr);
    if (F) {
        Launch l = cplx_launch(q->az, sizeof(C2<T>), (int)S2, B);
        k_cplx_synthesis<T, FAM_F, false><<<l.grid, l.block, l.smem, q->stream>>>(
            reinterpret_cast<const C2<T>*>(src), reinterpret_cast<C2<T>*>(q->X), S3, (int)S2, dev_axis<T>(q->az), none);
        s = check_launch(sl, "k_cplx_synthesis");
        if (s == HOBC_OK) s = vol_transpose<C2<T>>(q, q->X, sl->G, (int)S2, n0);
    } else {
        T* x = reinterpret_cast<T*>(q->X);
        switch (q->fam) {
            case FAM_S: s = pair_synthesis<T, FAM_S, 0>(sl, q->az, src, S3, n0, 1, x, S3, n0, (int)S2, B, none); break;
            case FAM_S3: s = pair_synthesis<T, FAM_S3, 0>(sl, q->az, src, S3, n0, 1, x, S3, n0, (int)S2, B, none); break;
            default: s = pair_synthesis<T, FAM_C, 0>(sl, q->az, src, S3, n0, 1, x, S3, n0, (int)S2, B, none); break;
        }
        if (s == HOBC_OK) s = vol_transpose<T>(q, q->X, sl->G, (int)S2, n0);
    }
    if (s != HOBC_OK) return s;
    return run_synthesis<T>(sl, sl->G, y);                          // slices [B][n0][S2] -> [B][n0][n1][n2]
}

template <typename T>
hobc_status run3_eig(hobc_volume_s* q, const void* psf, void* D) {
    hobc_plan_s* sl = q->slice;
    const AxisHost& a1 = sl->ax[0];
    const AxisHost& a2 = sl->ax[1];
    const int p0 = q->desc.psf[0];
    const long long S2 = (long long)q->S2, S3 = (long long)q->S3;
    const long long slice_psf = (long long)a1.p * a2.p;
    const dim3 g2((unsigned)(q->npsf * p0), (unsigned)a2.W);
    const dim3 g3((unsigned)S2, (unsigned)q->npsf);
    const int b3 = std::min(256, (q->az.n + 31) / 32 * 32);
    if (q->fam == FAM_F) {
        k_eig<T, true><<<g2, 256, 0, q->stream>>>(reinterpret_cast<const T*>(psf), slice_psf, a1.p, a2.p, a1.etab,
                                                  a2.etab, a1.etab2, a1.n, reinterpret_cast<C2<T>*>(q->D2), S2);
        k_vol_eig<T, true><<<g3, b3, 0, q->stream>>>(reinterpret_cast<const C2<T>*>(q->D2), p0, S2, q->az.etab,
                                                      q->az.n, reinterpret_cast<C2<T>*>(D), S3);
    } else {
        k_eig<T, false><<<g2, 256, 0, q->stream>>>(reinterpret_cast<const T*>(psf), slice_psf, a1.p, a2.p, a1.etab,
                                                   a2.etab, a1.etab2, a1.n, reinterpret_cast<T*>(q->D2), S2);
        k_vol_eig<T, false><<<g3, b3, 0, q->stream>>>(reinterpret_cast<const T*>(q->D2), p0, S2, q->az.etab,
                                                       q->az.n, reinterpret_cast<T*>(D), S3);
    }
    hobc_status s = check_launch(sl, "k_eig");
    if (s == HOBC_OK) ++sl->launches;
    return s;
}

template <typename T>
hobc_status run3_gcv(hobc_volume_s* q, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    hobc_plan_s* sl = q->slice;
    const GcvGeom geo = vol_geo<T>(q);
    const dim3 grid((unsigned)((long long)q->chunks * q->desc.batch));
    const size_t smem = 4 * (size_t)q->chunk * sizeof(T);
    if (q->fam == FAM_F)
        k_gcv_partials<T, true><<<grid, 256, smem, q->stream>>>(
            reinterpret_cast<const C2<T>*>(ghat), reinterpret_cast<const C2<T>*>(D), (long long)q->S3,
            q->desc.psf_per_item, reinterpret_cast<const T*>(sl->muT), geo, q->partials);
    else
        k_gcv_partials<T, false><<<grid, 256, smem, q->stream>>>(
            reinterpret_cast<const T*>(ghat), reinterpret_cast<const T*>(D), (long long)q->S3, q->desc.psf_per_item,
            reinterpret_cast<const T*>(sl->muT), geo, q->partials);
    hobc_status s = check_launch(sl, "k_gcv_partials");
    if (s != HOBC_OK) return s;
    cudaError_t e = launch_gcv_finalize_raw(q->partials, q->chunks, q->K, q->desc.batch, gcv, mu_idx, q->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error("k_gcv_finalize", e); return HOBC_ERR_CUDA; }
    ++sl->launches;
    return HOBC_OK;
}

}  // namespace hobc
