// The GCV curve of Eq. (eq:gcv2) by bin expansion (FP32 plans, 2D, one PSF for
// the batch; include/hobc.h, HOBC_GCV_EXPANSION).
//
// G(mu) = sum_i e_i/(a_i+mu)^2 / (sum_i w_i/(a_i+mu))^2 depends on an entry only
// through a_i = |d_i|^2/|s_i|^2 (eigenvalues and smoothing: the same for every
// image of the batch) and e_i = w_i |ghat_i|^2.  The entries are grouped by a:
// 256 bins uniform in log a over [a_lo, a_hi) = [1e-3 mu_min, 1e3 mu_max), a bin
// for a < a_lo and one for a >= a_hi.  In a bin of centre abar, with
// a = abar (1 + u) and rho = abar/(abar + mu),
//   1/(a+mu)   = 1/(abar+mu)   sum_p (-rho u)^p,
//   1/(a+mu)^2 = 1/(abar+mu)^2 sum_p (p+1) (-rho u)^p,
// so a bin contributes through the moments E_p = sum e u^p and W_p = sum w u^p,
// p = 0..7, and the curve costs bins x K evaluations instead of entries x K.
// Below a_lo the expansion is about 0 (u = a/a_lo, ratio a/mu <= 1e-3), above
// a_hi about infinity (u = a_hi/a, ratio mu/a <= 1e-3, the moments carry 1/a^2
// and 1/a).  The series is cut after p = 7: with bins of ratio r the inner bins
// have |rho u| <= U = sqrt(r) - 1, and every term keeps a relative error of at
// most 9 U^8/(1-U)^2 (the numerator's; 3.3e-9 for mu in [1e-8, 1], where
// r = 10^(14/256)), below the rounding of the FP32 sums.  Plans whose grid
// would make it exceed 1e-8 keep the direct scan.
//
// Per call: a key pass (bin and u of every entry, from the eigenvalues), a
// stable counting sort of the entries by bin, the moments of every piece of at
// most 256 entries of one bin (a warp each, FP32, fixed order), and per problem
// the sum of the pieces' moments (FP64, piece order), the curve (Horner in FP32,
// float-float sums over the bins) and its first minimum.  Every step runs in a
// fixed order: the result does not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hobc_internal.h"
#include "hobc_kernels.cuh"

namespace hobc {

static const int kGxBins = 256;               // inner bins, uniform in log a
static const int kGxKeys = kGxBins + 2;       // key 0: a < a_lo; 1..256 inner; 257: a >= a_hi
static const int kGxP = 8;                    // moments p = 0..7
static const int kGxChunk = 1024;             // entries per CTA of the key and scatter passes
static const int kGxPiece = 256;              // entries per piece (one warp)

struct GxTab {                                // bin geometry (device copy)
    float abar[kGxBins];                      // bin centres a_lo r^(b + 1/2)
    float inv_abar[kGxBins];
    float edge[kGxBins + 1];                  // bin edges a_lo r^b
    float a_lo, a_hi;
    float log2_alo, bins_per_log2;            // b = floor((log2 a - log2 a_lo) bins_per_log2)
};

}  // namespace hobc

struct hobc_gcvx_s {
    hobc::GxTab* tab;        // device
    int* key;                // [S] bin key of each stored entry (-1: dropped, s = 0)
    float* u;                // [S] expansion coordinate
    float* sn;               // [S] numerator scale (w, or w/a^2 above a_hi)
    float* sd;               // [S] denominator scale (w, or w/a above a_hi)
    int* s_idx;              // [S] the same four, sorted by key (stable)
    float* s_u;
    float* s_sn;
    float* s_sd;
    int* counts;             // [chunks][keys] entries per chunk and key, then their offsets
    int4* pieces;            // [max_pieces] start, length, key
    int* key_piece0;         // [keys + 1] first piece of each key; [keys] = number of pieces
    float* num_part;         // [batch][max_pieces][8]
    float* den_part;         // [max_pieces][8]
    int chunks, max_pieces;
    double bound;            // truncation bound of the series (relative, per term)
};

namespace hobc {

namespace {

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Bin key, expansion coordinate and scales of every stored entry; per-chunk key
// counts.  The GCV terms as in gcv_term: a = |d|^2/|s|^2 (capped), weight 2 for
// a Fourier entry that stands for a conjugate pair; entries with s = 0 dropped.
template <bool CPLX>
__global__ void __launch_bounds__(256)
k_gx_keys(const typename ElemT<float, CPLX>::t* __restrict__ D, GcvGeom geo, const GxTab* __restrict__ tab,
          long long S, int* __restrict__ key, float* __restrict__ u, float* __restrict__ sn,
          float* __restrict__ sd, int* __restrict__ counts) {
    __shared__ int hist[kGxKeys];
    for (int k = threadIdx.x; k < kGxKeys; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kGxChunk;
    const float a_lo = tab->a_lo, a_hi = tab->a_hi;
    for (int r = 0; r < kGxChunk / 256; ++r) {
        const long long i = base + r * 256 + threadIdx.x;
        if (i >= S) break;
        int c;
        const float s2 = lap_s2<float>(geo, i, c);
        float w = 1.f;
        if (CPLX) {
            const int nb = fam_nb(geo.fam), kk = c - nb;
            const bool self = (c < nb || c >= geo.W1 - nb || kk == 0 || 2 * kk == geo.N1);
            w = self ? 1.f : 2.f;
        }
        int k = -1;
        float uu = 0.f, vn = 0.f, vd = 0.f;
        if (s2 > 0.f) {
            const float a = fminf(abs2_of(D[i]) / s2, a_cap<float>());
            if (a < a_lo) {
                k = 0; uu = a / a_lo; vn = w; vd = w;
            } else if (a >= a_hi) {
                k = kGxKeys - 1; uu = a_hi / a; vd = w / a; vn = vd / a;
            } else {
                int b = (int)floorf((__log2f(a) - tab->log2_alo) * tab->bins_per_log2);
                b = max(0, min(kGxBins - 1, b));
                if (a < tab->edge[b] && b > 0) --b;                 // the approximate log2 may be one bin off
                else if (a >= tab->edge[b + 1] && b < kGxBins - 1) ++b;
                k = 1 + b;
                uu = (a - tab->abar[b]) * tab->inv_abar[b];
                vn = w; vd = w;
            }
            atomicAdd(&hist[k], 1);
        }
        key[i] = k; u[i] = uu; sn[i] = vn; sd[i] = vd;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kGxKeys; k += blockDim.x) counts[(long long)blockIdx.x * kGxKeys + k] = hist[k];
}

// Offsets of the stable counting sort (key-major, then chunk order) and the
// pieces: each key's range cut into pieces of at most kGxPiece entries.
// One CTA of 1024 threads.
__global__ void __launch_bounds__(1024)
k_gx_scan(int* __restrict__ counts, int chunks, int4* __restrict__ pieces, int* __restrict__ key_piece0) {
    __shared__ int tot[kGxKeys], start[kGxKeys], pstart[kGxKeys + 1];
    const int k = threadIdx.x;
    if (k < kGxKeys) {
        int t = 0;
        for (int c = 0; c < chunks; ++c) t += counts[(long long)c * kGxKeys + k];
        tot[k] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0, prun = 0;
        for (int j = 0; j < kGxKeys; ++j) {
            start[j] = run;
            pstart[j] = prun;
            run += tot[j];
            prun += (tot[j] + kGxPiece - 1) / kGxPiece;
        }
        pstart[kGxKeys] = prun;
    }
    __syncthreads();
    if (k < kGxKeys) {
        int run = start[k];
        for (int c = 0; c < chunks; ++c) {
            const long long o = (long long)c * kGxKeys + k;
            const int t = counts[o];
            counts[o] = run;
            run += t;
        }
        for (int q = 0; q * kGxPiece < tot[k]; ++q)
            pieces[pstart[k] + q] = make_int4(start[k] + q * kGxPiece, min(kGxPiece, tot[k] - q * kGxPiece), k, 0);
    }
    if (k <= kGxKeys) key_piece0[k] = pstart[k];
}

// Stable scatter into key order: warp w of a chunk owns entries
// [w 128, (w + 1) 128) of it; its entries of one key keep their index order
// (ranks from the lanes below with the same key, then a per-warp running count).
__global__ void __launch_bounds__(256)
k_gx_scatter(long long S, const int* __restrict__ key, const float* __restrict__ u, const float* __restrict__ sn,
             const float* __restrict__ sd, const int* __restrict__ offs, int* __restrict__ s_idx,
             float* __restrict__ s_u, float* __restrict__ s_sn, float* __restrict__ s_sd) {
    __shared__ int wc[8][kGxKeys];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < 8 * kGxKeys; j += blockDim.x) (&wc[0][0])[j] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kGxChunk + warp * (kGxChunk / 8);
    for (int it = 0; it < kGxChunk / 8 / 32; ++it) {          // counts per warp and key
        const long long i = base + it * 32 + lane;
        const int k = i < S ? key[i] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        if (k >= 0 && lane == __ffs(peers) - 1) wc[warp][k] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kGxKeys; k += blockDim.x) {  // exclusive prefix over the warps
        int run = 0;
        for (int w = 0; w < 8; ++w) {
            const int t = wc[w][k];
            wc[w][k] = run;
            run += t;
        }
    }
    __syncthreads();
    const int* off = offs + (long long)blockIdx.x * kGxKeys;
    for (int it = 0; it < kGxChunk / 8 / 32; ++it) {
        const long long i = base + it * 32 + lane;
        const int k = i < S ? key[i] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        if (k >= 0) {
            const int pos = off[k] + wc[warp][k] + __popc(peers & lanemask_lt());
            s_idx[pos] = (int)i;
            s_u[pos] = u[i];
            s_sn[pos] = sn[i];
            s_sd[pos] = sd[i];
        }
        __syncwarp();
        if (k >= 0 && lane == __ffs(peers) - 1) wc[warp][k] += __popc(peers);
        __syncwarp();
    }
}

// Moments sum_j v_j u_j^p, p = 0..7, of every piece: one warp per piece, each
// lane at most 8 entries in order, then a fixed shuffle tree.  NUM: v = sn |ghat|^2
// of problem blockIdx.y; else v = sd.
template <bool NUM, bool CPLX>
__global__ void __launch_bounds__(256)
k_gx_moments(const int4* __restrict__ pieces, const int* __restrict__ npieces, const int* __restrict__ s_idx,
             const float* __restrict__ s_u, const float* __restrict__ s_v,
             const typename ElemT<float, CPLX>::t* __restrict__ ghat, long long S, int max_pieces,
             float* __restrict__ part) {
    const int q = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (q >= *npieces) return;
    const long long item = blockIdx.y;
    const int4 pc = pieces[q];
    float m[kGxP];
#pragma unroll
    for (int p = 0; p < kGxP; ++p) m[p] = 0.f;
    for (int j = pc.x + lane; j < pc.x + pc.y; j += 32) {
        float t = s_v[j];
        if (NUM) t *= abs2_of(ghat[item * S + s_idx[j]]);
        const float uu = s_u[j];
#pragma unroll
        for (int p = 0; p < kGxP; ++p) {
            m[p] += t;
            t *= uu;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int p = 0; p < kGxP; ++p) m[p] += __shfl_down_sync(0xffffffffu, m[p], off);
    if (lane == 0) {
        float4* o = reinterpret_cast<float4*>(part + ((long long)item * max_pieces + q) * kGxP);
        o[0] = make_float4(m[0], m[1], m[2], m[3]);
        o[1] = make_float4(m[4], m[5], m[6], m[7]);
    }
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bv = __fsub_rn(s, hi);
    lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(x, bv));
    hi = s;
}

// Per problem: the moments of every key (FP64 over its pieces, in order), the
// curve G(mu_j) and its first minimum (NaN never wins).  One CTA per problem.
__global__ void __launch_bounds__(256)
k_gx_finalize(const float* __restrict__ num_part, const float* __restrict__ den_part,
              const int* __restrict__ key_piece0, const GxTab* __restrict__ tab, const double* __restrict__ mu,
              int K, int max_pieces, double* __restrict__ gcv, int* __restrict__ mu_idx) {
    __shared__ float Ec[kGxKeys][kGxP];     // (p + 1) E_p
    __shared__ float Wc[kGxKeys][kGxP];
    __shared__ int kp0[kGxKeys + 1];
    __shared__ double rbest[256];
    __shared__ int ridx[256];
    const long long item = blockIdx.x;
    for (int k = threadIdx.x; k <= kGxKeys; k += blockDim.x) kp0[k] = key_piece0[k];
    __syncthreads();
    for (int kp = threadIdx.x; kp < kGxKeys * kGxP; kp += blockDim.x) {
        const int k = kp / kGxP, p = kp - k * kGxP;
        double se = 0, sw = 0;
        for (int q = kp0[k]; q < kp0[k + 1]; ++q) {
            se += (double)num_part[((long long)item * max_pieces + q) * kGxP + p];
            sw += (double)den_part[(long long)q * kGxP + p];
        }
        Ec[k][p] = (float)(se * (p + 1));
        Wc[k][p] = (float)sw;
    }
    __syncthreads();
    const float a_lo = tab->a_lo, a_hi = tab->a_hi;
    double best = 0;
    int bi = 0x7fffffff;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        const float m = (float)mu[j];
        float nh = 0, nl = 0, dh = 0, dl = 0;
        for (int k = 0; k < kGxKeys; ++k) {
            if (kp0[k] == kp0[k + 1]) continue;
            float x, sn_, sd_;
            if (k == 0) {
                const float inv = 1.f / m;
                x = -a_lo * inv; sn_ = inv * inv; sd_ = inv;
            } else if (k == kGxKeys - 1) {
                x = -m / a_hi; sn_ = 1.f; sd_ = 1.f;
            } else {
                const float ab = tab->abar[k - 1];
                const float inv = 1.f / (ab + m);
                x = -ab * inv; sn_ = inv * inv; sd_ = inv;
            }
            float hn = Ec[k][kGxP - 1], hd = Wc[k][kGxP - 1];
#pragma unroll
            for (int p = kGxP - 2; p >= 0; --p) {
                hn = fmaf(hn, x, Ec[k][p]);
                hd = fmaf(hd, x, Wc[k][p]);
            }
            two_sum_acc(nh, nl, hn * sn_);
            two_sum_acc(dh, dl, hd * sd_);
        }
        const double den = (double)dh + (double)dl;
        const double G = ((double)nh + (double)nl) / (den * den);
        if (gcv) gcv[item * K + j] = G;
        if (!isnan(G) && (bi == 0x7fffffff || G < best)) { best = G; bi = j; }
    }
    rbest[threadIdx.x] = best;
    ridx[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double ob = rbest[threadIdx.x + s];
            const int oi = ridx[threadIdx.x + s];
            const int ci = ridx[threadIdx.x];
            if (oi != 0x7fffffff && (ci == 0x7fffffff || ob < rbest[threadIdx.x] ||
                                     (ob == rbest[threadIdx.x] && oi < ci))) {
                rbest[threadIdx.x] = ob;
                ridx[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) mu_idx[item] = ridx[0] == 0x7fffffff ? 0 : ridx[0];
}

}  // namespace

void gcvx_free(hobc_plan_s* p) {
    hobc_gcvx_s* x = p->gx;
    if (!x) return;
    cudaFree(x->tab); cudaFree(x->key); cudaFree(x->u); cudaFree(x->sn); cudaFree(x->sd);
    cudaFree(x->s_idx); cudaFree(x->s_u); cudaFree(x->s_sn); cudaFree(x->s_sd);
    cudaFree(x->counts); cudaFree(x->pieces); cudaFree(x->key_piece0); cudaFree(x->num_part); cudaFree(x->den_part);
    delete x;
    p->gx = nullptr;
}

// Truncation bound of the series for a grid [mu_min, mu_max] (relative error of
// a numerator term; the denominator's is smaller): 9 U^8/(1-U)^2 with U the
// largest |rho u| of an inner bin (and 9 (1e-3)^8 for the outer keys).
static double gx_bound(double mu_min, double mu_max, double* r_out) {
    const double decades = std::log10(mu_max / mu_min) + 6.0;
    const double r = std::pow(10.0, decades / kGxBins);
    const double U = std::sqrt(r) - 1.0 + 1e-6;             // margin for the rounding of the edges
    if (r_out) *r_out = r;
    return std::max(9.0 * std::pow(U, 8) / ((1 - U) * (1 - U)), 9.0 * std::pow(1e-3, 8));
}

static hobc_status gcvx_prepare(hobc_plan_s* p) {
    std::vector<double> mu(p->K);
    cudaError_t e = cudaMemcpy(mu.data(), p->mu, sizeof(double) * p->K, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_last_error("hobc_plan_set_gcv_mode", e); return HOBC_ERR_CUDA; }
    const double mu_min = *std::min_element(mu.begin(), mu.end());
    const double mu_max = *std::max_element(mu.begin(), mu.end());
    double r = 0;
    const double bound = gx_bound(mu_min, mu_max, &r);
    if (!(bound <= 1e-8)) {
        char msg[200];
        snprintf(msg, sizeof(msg), "hobc_plan_set_gcv_mode: the mu grid spans too many decades for the "
                                   "expansion (bound %.2e > 1e-8)", bound);
        set_last_error_text(msg);
        return HOBC_ERR_UNSUPPORTED;
    }
    GxTab t;
    memset(&t, 0, sizeof(t));
    const double a_lo = 1e-3 * mu_min, a_hi = 1e3 * mu_max;
    for (int b = 0; b <= kGxBins; ++b) t.edge[b] = (float)(a_lo * std::pow(r, b));
    for (int b = 0; b < kGxBins; ++b) {
        const double ab = a_lo * std::pow(r, b + 0.5);
        t.abar[b] = (float)ab;
        t.inv_abar[b] = (float)(1.0 / ab);
    }
    t.a_lo = (float)a_lo;
    t.a_hi = (float)t.edge[kGxBins];
    t.log2_alo = (float)std::log2(a_lo);
    t.bins_per_log2 = (float)(1.0 / std::log2(r));
    hobc_gcvx_s* x = new hobc_gcvx_s();
    memset(x, 0, sizeof(*x));
    p->gx = x;
    const size_t S = p->spec_elems;
    x->chunks = (int)((S + kGxChunk - 1) / kGxChunk);
    x->max_pieces = (int)((S + kGxPiece - 1) / kGxPiece) + kGxKeys;
    x->bound = bound;
    auto alloc = [&](void** ptr, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(ptr, bytes); };
    alloc((void**)&x->tab, sizeof(GxTab));
    alloc((void**)&x->key, S * sizeof(int));
    alloc((void**)&x->u, S * sizeof(float));
    alloc((void**)&x->sn, S * sizeof(float));
    alloc((void**)&x->sd, S * sizeof(float));
    alloc((void**)&x->s_idx, S * sizeof(int));
    alloc((void**)&x->s_u, S * sizeof(float));
    alloc((void**)&x->s_sn, S * sizeof(float));
    alloc((void**)&x->s_sd, S * sizeof(float));
    alloc((void**)&x->counts, (size_t)x->chunks * kGxKeys * sizeof(int));
    alloc((void**)&x->pieces, (size_t)x->max_pieces * sizeof(int4));
    alloc((void**)&x->key_piece0, (kGxKeys + 1) * sizeof(int));
    alloc((void**)&x->num_part, (size_t)p->desc.batch * x->max_pieces * kGxP * sizeof(float));
    alloc((void**)&x->den_part, (size_t)x->max_pieces * kGxP * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(x->tab, &t, sizeof(t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_last_error("hobc_plan_set_gcv_mode", e);
        gcvx_free(p);
        return HOBC_ERR_CUDA;
    }
    return HOBC_OK;
}

static hobc_status gx_check(hobc_plan_s* p, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(what, e);
        return HOBC_ERR_CUDA;
    }
    ++p->launches;
    return HOBC_OK;
}

template <bool CPLX>
static hobc_status gcvx_launch(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    typedef typename ElemT<float, CPLX>::t E;
    hobc_gcvx_s* x = p->gx;
    GcvGeom geo;
    memset(&geo, 0, sizeof(geo));
    geo.ndim = 2;
    geo.fam = p->fam;
    geo.n0 = p->ax[0].n; geo.N0 = p->ax[0].N;
    geo.n1 = p->ax[1].n; geo.N1 = p->ax[1].N; geo.W1 = p->ax[1].W;
    geo.lap = p->desc.L == HOBC_L_LAPLACIAN;
    geo.S = (long long)p->spec_elems;
    geo.K = p->K;
    const long long S = geo.S;
    cudaStream_t st = p->stream;
    k_gx_keys<CPLX><<<x->chunks, 256, 0, st>>>(reinterpret_cast<const E*>(D), geo, x->tab, S, x->key, x->u, x->sn,
                                                x->sd, x->counts);
    hobc_status s = gx_check(p, "k_gx_keys");
    if (s != HOBC_OK) return s;
    k_gx_scan<<<1, 1024, 0, st>>>(x->counts, x->chunks, x->pieces, x->key_piece0);
    if ((s = gx_check(p, "k_gx_scan")) != HOBC_OK) return s;
    k_gx_scatter<<<x->chunks, 256, 0, st>>>(S, x->key, x->u, x->sn, x->sd, x->counts, x->s_idx, x->s_u, x->s_sn,
                                            x->s_sd);
    if ((s = gx_check(p, "k_gx_scatter")) != HOBC_OK) return s;
    const dim3 g1((x->max_pieces + 7) / 8, 1), gB((x->max_pieces + 7) / 8, p->desc.batch);
    k_gx_moments<false, CPLX><<<g1, 256, 0, st>>>(x->pieces, x->key_piece0 + kGxKeys, x->s_idx, x->s_u, x->s_sd,
                                                   nullptr, S, x->max_pieces, x->den_part);
    if ((s = gx_check(p, "k_gx_moments")) != HOBC_OK) return s;
    k_gx_moments<true, CPLX><<<gB, 256, 0, st>>>(x->pieces, x->key_piece0 + kGxKeys, x->s_idx, x->s_u, x->s_sn,
                                                  reinterpret_cast<const E*>(ghat), S, x->max_pieces, x->num_part);
    if ((s = gx_check(p, "k_gx_moments")) != HOBC_OK) return s;
    k_gx_finalize<<<p->desc.batch, 256, 0, st>>>(x->num_part, x->den_part, x->key_piece0, x->tab, p->mu, p->K,
                                                 x->max_pieces, gcv, mu_idx);
    return gx_check(p, "k_gx_finalize");
}

bool gcvx_active(const hobc_plan_s* p) { return p->gcv_mode == HOBC_GCV_EXPANSION && p->gx != nullptr; }

hobc_status run_gcv_expansion(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    return fam_fourier(p->fam) ? gcvx_launch<true>(p, ghat, D, gcv, mu_idx)
                               : gcvx_launch<false>(p, ghat, D, gcv, mu_idx);
}

}  // namespace hobc

using namespace hobc;

extern "C" {

hobc_status hobc_plan_set_gcv_mode(hobc_plan* p, int mode) {
    if (!p) return HOBC_ERR_ARG;
    if (mode == HOBC_GCV_DIRECT) {
        p->gcv_mode = HOBC_GCV_DIRECT;
        return HOBC_OK;
    }
    if (mode != HOBC_GCV_EXPANSION) return HOBC_ERR_ARG;
    if (p->prec == HOBC_FP64 || p->nax != 2 || p->desc.psf_per_item) {
        set_last_error_text("hobc_plan_set_gcv_mode: the expansion serves FP32 and split-BF16 2D plans "
                            "with one PSF for the batch");
        return HOBC_ERR_UNSUPPORTED;
    }
    if (!p->gx) {
        const hobc_status s = gcvx_prepare(p);
        if (s != HOBC_OK) return s;
    }
    p->gcv_mode = HOBC_GCV_EXPANSION;
    return HOBC_OK;
}

int hobc_plan_gcv_mode(const hobc_plan* p) { return p ? p->gcv_mode : -1; }

double hobc_gcv_expansion_bound(const hobc_plan* p) { return (p && p->gx) ? p->gx->bound : -1.0; }

}  // extern "C"
