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
// most 256 entries of one bin (a warp each, FP32, fixed order), per key and
// problem the sum of its pieces' moments (FP64, fixed order), the curve (Horner
// in FP32, float-float sums over the bins; a CTA per 32 grid values and
// problem) and each problem's first minimum.  Every step runs in a fixed order: the result does not depend on
// scheduling.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hobc_internal.h"
#include "hobc_gcvx.cuh"

namespace hobc {

static const int kGxChunk = 1024;             // entries per CTA of the key and scatter passes
static const int kGxPiece = 256;              // entries per piece (one warp)
static const int kGxIpw = 4;                  // problems per warp of the moments pass

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
    int* counts;             // [keys][chunks] entries per key and chunk, then their prefix within the key
    int* tot;                // [keys] entries per key
    int* key_start;          // [keys] first sorted position of each key
    float2* gmom;            // [batch + 1][max_groups][8] moments per piece group, float-float (numerators, then the denominator's)
    float2* kmom;            // [batch + 1][keys][8] moments per key, float-float
    double* G_ws;            // [batch][K] the curve
    int4* groups;            // [max_groups] first piece, pieces, key
    int* key_group0;         // [keys + 1] first group of each key; [keys] = number of groups
    unsigned* done;          // [1 + batch] completion counters (chunk scan, then one per problem's curve)
    int4* pieces;            // [max_pieces] start, length, key
    int* key_piece0;         // [keys + 1] first piece of each key; [keys] = number of pieces
    float* num_part;         // [batch][max_pieces][8]
    float* den_part;         // [max_pieces][8]
    int chunks, max_pieces, max_groups;
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
            k = gx_classify(a, w, tab, uu, vn, vd);
            atomicAdd(&hist[k], 1);
        }
        key[i] = k; u[i] = uu; sn[i] = vn; sd[i] = vd;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kGxKeys; k += blockDim.x) counts[(long long)k * gridDim.x + blockIdx.x] = hist[k];
}

// Start of every key in the sorted order, its pieces (its range cut into
// pieces of at most kGxPiece entries) and its piece groups (at most 32 pieces
// each), from the key totals.  Run by one CTA of 256 threads.
__device__ void gx_scan_body(const int* __restrict__ tot, int* __restrict__ key_start, int4* __restrict__ pieces,
                             int* __restrict__ key_piece0, int4* __restrict__ groups, int* __restrict__ key_group0) {
    __shared__ int st[kGxKeys], tt[kGxKeys], ps[kGxKeys + 1], gs[kGxKeys + 1];
    __shared__ int wsum[8][3];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // thread t holds keys 2t, 2t + 1 (129 threads): entries, pieces and groups,
    // then an exclusive scan over the threads (warp shuffles, then the warp totals)
    int e[2] = {0, 0}, pc[2] = {0, 0}, gc[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (2 * t + h < kGxKeys) {
            e[h] = __ldcg(tot + 2 * t + h);
            pc[h] = (e[h] + kGxPiece - 1) / kGxPiece;
            gc[h] = (pc[h] + 31) / 32;
            tt[2 * t + h] = e[h];
        }
    int x[3] = {e[0] + e[1], pc[0] + pc[1], gc[0] + gc[1]};
    const int own[3] = {x[0], x[1], x[2]};
#pragma unroll
    for (int off = 1; off < 32; off <<= 1)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const int y = __shfl_up_sync(0xffffffffu, x[v], off);
            if (lane >= off) x[v] += y;
        }
    if (lane == 31)
#pragma unroll
        for (int v = 0; v < 3; ++v) wsum[warp][v] = x[v];
    __syncthreads();
    int ex[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        int base = 0;
        for (int w = 0; w < warp; ++w) base += wsum[w][v];
        ex[v] = base + x[v] - own[v];
    }
    if (2 * t < kGxKeys) { st[2 * t] = ex[0]; ps[2 * t] = ex[1]; gs[2 * t] = ex[2]; }
    if (2 * t + 1 < kGxKeys) { st[2 * t + 1] = ex[0] + e[0]; ps[2 * t + 1] = ex[1] + pc[0]; gs[2 * t + 1] = ex[2] + gc[0]; }
    if (2 * t + 1 == kGxKeys - 1) { ps[kGxKeys] = ex[1] + own[1]; gs[kGxKeys] = ex[2] + own[2]; }
    __syncthreads();
    for (int k = t; k < kGxKeys; k += blockDim.x) key_start[k] = st[k];
    for (int k = t; k <= kGxKeys; k += blockDim.x) { key_piece0[k] = ps[k]; key_group0[k] = gs[k]; }
    for (int q = t; q < ps[kGxKeys]; q += blockDim.x) {
        int lo = 0, hi = kGxKeys - 1;               // the key whose pieces hold q
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ps[mid] <= q) lo = mid; else hi = mid - 1;
        }
        const int r = q - ps[lo];
        pieces[q] = make_int4(st[lo] + r * kGxPiece, min(kGxPiece, tt[lo] - r * kGxPiece), lo, 0);
    }
    for (int g = t; g < gs[kGxKeys]; g += blockDim.x) {
        int lo = 0, hi = kGxKeys - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (gs[mid] <= g) lo = mid; else hi = mid - 1;
        }
        const int r = g - gs[lo];
        const int q0 = ps[lo] + 32 * r;
        groups[g] = make_int4(q0, min(32, ps[lo + 1] - q0), lo, 0);
    }
}

// Per key, the exclusive prefix of its counts over the chunks (in place) and
// its total: one warp per key.  The CTA that
// finishes last (a counter, reset by it) then runs gx_scan_body.
__global__ void __launch_bounds__(256)
k_gx_chunkscan(int* __restrict__ counts, int chunks, int* __restrict__ tot, unsigned* __restrict__ done,
               int* __restrict__ key_start, int4* __restrict__ pieces, int* __restrict__ key_piece0,
               int4* __restrict__ groups, int* __restrict__ key_group0) {
    __shared__ bool last;
    const int k = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k < kGxKeys) {
        // tiles of 1024 chunks: lane l holds chunks 32 l .. 32 l + 31 of the tile
        // (loaded together), its own running sum, then a scan over the lanes
        int run = 0;
        int* row = counts + (long long)k * chunks;
        for (int t0 = 0; t0 < chunks; t0 += 1024) {
            int v[32];
            const int c0 = t0 + 32 * lane;
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = c0 + i < chunks ? row[c0 + i] : 0;
            int own = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) { const int t = v[i]; v[i] = own; own += t; }
            int x = own;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += y;
            }
            const int base = run + x - own;
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (c0 + i < chunks) row[c0 + i] = base + v[i];
            run += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) tot[k] = run;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    gx_scan_body(tot, key_start, pieces, key_piece0, groups, key_group0);
    if (threadIdx.x == 0) *done = 0;
}

// Stable scatter into key order: warp w of a chunk owns entries
// [w 128, (w + 1) 128) of it; its entries of one key keep their index order
// (ranks from the lanes below with the same key, then a per-warp running count).
__global__ void __launch_bounds__(256)
k_gx_scatter(long long S, const int* __restrict__ key, const float* __restrict__ u, const float* __restrict__ sn,
             const float* __restrict__ sd, const int* __restrict__ offs, const int* __restrict__ key_start,
             int* __restrict__ s_idx,
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
    const int* off = offs + blockIdx.x;          // offs[k * chunks + chunk]
    const long long kstride = gridDim.x;
    for (int it = 0; it < kGxChunk / 8 / 32; ++it) {
        const long long i = base + it * 32 + lane;
        const int k = i < S ? key[i] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        if (k >= 0) {
            const int pos = key_start[k] + off[k * kstride] + wc[warp][k] + __popc(peers & lanemask_lt());
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
// lane at most 8 entries (held in registers across the kGxIpw problems of grid
// row y), summed in entry order, then a fixed shuffle tree.  Rows y < num_rows:
// v = sn |ghat|^2 of each problem in turn; a row past them: v = sd.
template <bool CPLX>
__global__ void __launch_bounds__(256, 5)
k_gx_moments(const int4* __restrict__ pieces, const int* __restrict__ npieces, const int* __restrict__ s_idx,
             const float* __restrict__ s_u, const float* __restrict__ s_sn, const float* __restrict__ s_sd,
             const typename ElemT<float, CPLX>::t* __restrict__ ghat, long long S, int items, int num_rows,
             int max_pieces, float* __restrict__ num_part, float* __restrict__ den_part) {
    constexpr int E = kGxPiece / 32;
    const int q = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (q >= *npieces) return;
    const bool NUM = (int)blockIdx.y < num_rows;                 // rows past num_rows: the denominator's moments
    const float* s_v = NUM ? s_sn : s_sd;
    float* part = NUM ? num_part : den_part;
    const int4 pc = pieces[q];
    int id[E];
    float uu[E], vv[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int j = pc.x + lane + 32 * m;
        const bool in = lane + 32 * m < pc.y;
        id[m] = in ? (NUM ? s_idx[j] : 0) : -1;
        uu[m] = in ? s_u[j] : 0.f;
        vv[m] = in ? s_v[j] : 0.f;
    }
    const int item0 = NUM ? blockIdx.y * kGxIpw : 0;
    const int nit = NUM ? min(items - item0, kGxIpw) : 1;
    for (int it = 0; it < nit; ++it) {
        const int item = item0 + it;
        float g2[E];
#pragma unroll
        for (int m = 0; m < E; ++m)
            g2[m] = (NUM && id[m] >= 0) ? abs2_of(ghat[(long long)item * S + id[m]]) : 1.f;
        float mo[kGxP];
#pragma unroll
        for (int p = 0; p < kGxP; ++p) mo[p] = 0.f;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            float t = vv[m] * g2[m];
#pragma unroll
            for (int p = 0; p < kGxP; ++p) {
                mo[p] += t;
                t *= uu[m];
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int p = 0; p < kGxP; ++p) mo[p] += __shfl_down_sync(0xffffffffu, mo[p], off);
        if (lane == 0) {
            float4* o = reinterpret_cast<float4*>(part + ((long long)item * max_pieces + q) * kGxP);
            o[0] = make_float4(mo[0], mo[1], mo[2], mo[3]);
            o[1] = make_float4(mo[4], mo[5], mo[6], mo[7]);
        }
    }
}

// The moments of every piece group: the sum over its (at most 32) pieces in
// float-float, lane l taking piece l, then a fixed shuffle tree.  Grid y <
// batch: the numerator moments of problem y; y = batch: the denominator's.
__global__ void __launch_bounds__(256)
k_gx_reduce(const float* __restrict__ num_part, const float* __restrict__ den_part, const int4* __restrict__ groups,
            const int* __restrict__ ngroups, int batch, int max_pieces, int max_groups, float2* __restrict__ gmom) {
    const int g = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31, y = blockIdx.y;
    if (g >= *ngroups) return;
    const int4 gr = groups[g];
    const float* src = y < batch ? num_part + (long long)y * max_pieces * kGxP : den_part;
    float hi[kGxP], lo[kGxP];
#pragma unroll
    for (int p = 0; p < kGxP; ++p) { hi[p] = 0.f; lo[p] = 0.f; }
    if (lane < gr.y) {
        const float4 a = reinterpret_cast<const float4*>(src + (long long)(gr.x + lane) * kGxP)[0];
        const float4 b = reinterpret_cast<const float4*>(src + (long long)(gr.x + lane) * kGxP)[1];
        hi[0] = a.x; hi[1] = a.y; hi[2] = a.z; hi[3] = a.w;
        hi[4] = b.x; hi[5] = b.y; hi[6] = b.z; hi[7] = b.w;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int p = 0; p < kGxP; ++p) {
            const float oh = __shfl_down_sync(0xffffffffu, hi[p], off);
            const float ol = __shfl_down_sync(0xffffffffu, lo[p], off);
            two_sum_acc(hi[p], lo[p], oh);
            lo[p] += ol;
        }
    if (lane == 0)
#pragma unroll
        for (int p = 0; p < kGxP; ++p) gmom[((long long)y * max_groups + g) * kGxP + p] = make_float2(hi[p], lo[p]);
}

// The moments of every key: the sum over its groups in float-float, lane l
// taking groups l, l + 32, ... in order, then a fixed shuffle tree.  Grid y as
// for k_gx_reduce.
__global__ void __launch_bounds__(256)
k_gx_keysum(const float2* __restrict__ gmom, const int* __restrict__ key_group0, int max_groups,
            float2* __restrict__ kmom) {
    const int k = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31, y = blockIdx.y;
    if (k >= kGxKeys) return;
    const int g0 = key_group0[k], g1 = key_group0[k + 1];
    float hi[kGxP], lo[kGxP];
#pragma unroll
    for (int p = 0; p < kGxP; ++p) { hi[p] = 0.f; lo[p] = 0.f; }
    for (int g = g0 + lane; g < g1; g += 32)
#pragma unroll
        for (int p = 0; p < kGxP; ++p) {
            const float2 v = gmom[((long long)y * max_groups + g) * kGxP + p];
            two_sum_acc(hi[p], lo[p], v.x);
            lo[p] += v.y;
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int p = 0; p < kGxP; ++p) {
            const float oh = __shfl_down_sync(0xffffffffu, hi[p], off);
            const float ol = __shfl_down_sync(0xffffffffu, lo[p], off);
            two_sum_acc(hi[p], lo[p], oh);
            lo[p] += ol;
        }
    if (lane == 0)
#pragma unroll
        for (int p = 0; p < kGxP; ++p) kmom[((long long)y * kGxKeys + k) * kGxP + p] = make_float2(hi[p], lo[p]);
}

// The curve: block (mu group of 32, problem), from the moments of every key; thread (slice, j) sums the keys slice, slice + 8,
// ... at grid value j (Horner in FP32, float-float sums), and the 8 slices are
// added in order; G = num / den^2 in double.  The CTA that completes a problem's
// curve last takes its first minimum (NaN never wins).
__global__ void __launch_bounds__(256)
k_gx_curve(const float2* __restrict__ kmom, int batch, const int* __restrict__ key_group0,
           const GxTab* __restrict__ tab, const double* __restrict__ mu, int K, double* __restrict__ G_ws,
           double* __restrict__ gcv, unsigned* __restrict__ done, int* __restrict__ mu_idx) {
    __shared__ float Ec[kGxKeys][kGxP];     // (p + 1) E_p
    __shared__ float Wc[kGxKeys][kGxP];
    __shared__ int nonempty[kGxKeys];
    __shared__ float red[4][8][32];
    const long long item = blockIdx.y;
    constexpr int kLoads = (kGxKeys * kGxP + 255) / 256;
    float2 va[kLoads], vb[kLoads];              // all loads first (the block has 256 threads)
#pragma unroll
    for (int i = 0; i < kLoads; ++i) {
        const int kp = threadIdx.x + 256 * i;
        if (kp < kGxKeys * kGxP) {
            va[i] = kmom[item * kGxKeys * kGxP + kp];
            vb[i] = kmom[(long long)batch * kGxKeys * kGxP + kp];
        }
    }
#pragma unroll
    for (int i = 0; i < kLoads; ++i) {
        const int kp = threadIdx.x + 256 * i;
        if (kp < kGxKeys * kGxP) {
            (&Ec[0][0])[kp] = (va[i].x + va[i].y) * (float)(kp % kGxP + 1);
            (&Wc[0][0])[kp] = vb[i].x + vb[i].y;
        }
    }
    for (int k = threadIdx.x; k < kGxKeys; k += blockDim.x) nonempty[k] = key_group0[k] != key_group0[k + 1];
    __syncthreads();
    const int jl = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + jl;
    const float m = j < K ? (float)mu[j] : 1.f;
    float nh = 0, nl = 0, dh = 0, dl = 0;
    for (int k = slice; k < kGxKeys; k += 8) {
        if (!nonempty[k]) continue;
        float x, sn_, sd_;
        gx_key_terms(k, m, tab, x, sn_, sd_);
        float hn = Ec[k][kGxP - 1], hd = Wc[k][kGxP - 1];
#pragma unroll
        for (int p = kGxP - 2; p >= 0; --p) {
            hn = fmaf(hn, x, Ec[k][p]);
            hd = fmaf(hd, x, Wc[k][p]);
        }
        two_sum_acc(nh, nl, hn * sn_);
        two_sum_acc(dh, dl, hd * sd_);
    }
    red[0][slice][jl] = nh; red[1][slice][jl] = nl; red[2][slice][jl] = dh; red[3][slice][jl] = dl;
    __syncthreads();
    if (slice == 0 && j < K) {
        float ah = 0, al = 0, bh = 0, bl = 0;
        for (int sl = 0; sl < 8; ++sl) {
            two_sum_acc(ah, al, red[0][sl][jl]);
            al += red[1][sl][jl];
            two_sum_acc(bh, bl, red[2][sl][jl]);
            bl += red[3][sl][jl];
        }
        const double den = (double)bh + (double)bl;
        const double Gj = ((double)ah + (double)al) / (den * den);
        G_ws[item * K + j] = Gj;
        if (gcv) gcv[item * K + j] = Gj;
    }
    // the CTA that finishes this problem's curve last takes its first minimum
    __shared__ bool last;
    __shared__ double rbest[256];
    __shared__ int ridx[256];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done + item, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double best = 0;
    int bi = 0x7fffffff;
    for (int jj = threadIdx.x; jj < K; jj += blockDim.x) {
        const double G = __ldcg(G_ws + item * K + jj);
        if (!isnan(G) && (bi == 0x7fffffff || G < best)) { best = G; bi = jj; }
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
    if (threadIdx.x == 0) {
        mu_idx[item] = ridx[0] == 0x7fffffff ? 0 : ridx[0];
        done[item] = 0;
    }
}

}  // namespace

void gcvx_free(hobc_plan_s* p) {
    hobc_gcvx_s* x = p->gx;
    if (!x) return;
    cudaFree(x->tab); cudaFree(x->key); cudaFree(x->u); cudaFree(x->sn); cudaFree(x->sd);
    cudaFree(x->s_idx); cudaFree(x->s_u); cudaFree(x->s_sn); cudaFree(x->s_sd);
    cudaFree(x->counts); cudaFree(x->tot); cudaFree(x->key_start); cudaFree(x->gmom); cudaFree(x->kmom); cudaFree(x->G_ws); cudaFree(x->groups);
    cudaFree(x->key_group0); cudaFree(x->done); cudaFree(x->pieces); cudaFree(x->key_piece0); cudaFree(x->num_part); cudaFree(x->den_part);
    delete x;
    p->gx = nullptr;
}

static hobc_status gcvx_setup(hobc_plan_s* p) {
    std::vector<double> mu(p->K);
    cudaError_t e = cudaMemcpy(mu.data(), p->mu, sizeof(double) * p->K, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_last_error("hobc_plan_set_gcv_mode", e); return HOBC_ERR_CUDA; }
    GxTab t;
    double bound = 0;
    gx_make_table(mu.data(), p->K, t, &bound);
    if (!(bound <= 1e-8)) {
        char msg[200];
        snprintf(msg, sizeof(msg), "hobc_plan_set_gcv_mode: the mu grid spans too many decades for the "
                                   "expansion (bound %.2e > 1e-8)", bound);
        set_last_error_text(msg);
        return HOBC_ERR_UNSUPPORTED;
    }
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
    alloc((void**)&x->tot, kGxKeys * sizeof(int));
    alloc((void**)&x->key_start, kGxKeys * sizeof(int));
    x->max_groups = x->max_pieces / 32 + kGxKeys + 1;
    alloc((void**)&x->gmom, (size_t)(p->desc.batch + 1) * x->max_groups * kGxP * sizeof(float2));
    alloc((void**)&x->groups, (size_t)x->max_groups * sizeof(int4));
    alloc((void**)&x->kmom, (size_t)(p->desc.batch + 1) * kGxKeys * kGxP * sizeof(float2));
    alloc((void**)&x->key_group0, (kGxKeys + 1) * sizeof(int));
    alloc((void**)&x->done, (size_t)(p->desc.batch + 1) * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(x->done, 0, (size_t)(p->desc.batch + 1) * sizeof(unsigned));
    alloc((void**)&x->G_ws, (size_t)p->desc.batch * p->K * sizeof(double));
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

// The steps that depend on the eigenvalues alone: keys, the counting sort and
// the denominator's piece moments.
template <bool CPLX>
static hobc_status gcvx_prepare_d(hobc_plan_s* p, const void* D) {
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
    k_gx_chunkscan<<<(kGxKeys + 7) / 8, 256, 0, st>>>(x->counts, x->chunks, x->tot, x->done, x->key_start,
                                                      x->pieces, x->key_piece0, x->groups, x->key_group0);
    if ((s = gx_check(p, "k_gx_chunkscan")) != HOBC_OK) return s;
    k_gx_scatter<<<x->chunks, 256, 0, st>>>(S, x->key, x->u, x->sn, x->sd, x->counts, x->key_start, x->s_idx,
                                            x->s_u, x->s_sn, x->s_sd);
    if ((s = gx_check(p, "k_gx_scatter")) != HOBC_OK) return s;
    k_gx_moments<CPLX><<<dim3((x->max_pieces + 7) / 8, 1), 256, 0, st>>>(
        x->pieces, x->key_piece0 + kGxKeys, x->s_idx, x->s_u, x->s_sn, x->s_sd, nullptr, S, 0, 0, x->max_pieces,
        x->num_part, x->den_part);
    return gx_check(p, "k_gx_moments");
}

// The steps of each batch of spectra: the numerators' piece moments, the group
// and key sums and the curve.
template <bool CPLX>
static hobc_status gcvx_curves(hobc_plan_s* p, const void* ghat, double* gcv, int* mu_idx) {
    typedef typename ElemT<float, CPLX>::t E;
    hobc_gcvx_s* x = p->gx;
    const long long S = (long long)p->spec_elems;
    cudaStream_t st = p->stream;
    const int B = p->desc.batch;
    const int rows = (B + kGxIpw - 1) / kGxIpw;
    k_gx_moments<CPLX><<<dim3((x->max_pieces + 7) / 8, rows), 256, 0, st>>>(
        x->pieces, x->key_piece0 + kGxKeys, x->s_idx, x->s_u, x->s_sn, x->s_sd, reinterpret_cast<const E*>(ghat), S,
        B, rows, x->max_pieces, x->num_part, x->den_part);
    hobc_status s = gx_check(p, "k_gx_moments");
    if (s != HOBC_OK) return s;
    k_gx_reduce<<<dim3((x->max_groups + 7) / 8, B + 1), 256, 0, st>>>(
        x->num_part, x->den_part, x->groups, x->key_group0 + kGxKeys, B, x->max_pieces, x->max_groups, x->gmom);
    if ((s = gx_check(p, "k_gx_reduce")) != HOBC_OK) return s;
    k_gx_keysum<<<dim3((kGxKeys + 7) / 8, B + 1), 256, 0, st>>>(x->gmom, x->key_group0, x->max_groups, x->kmom);
    if ((s = gx_check(p, "k_gx_keysum")) != HOBC_OK) return s;
    k_gx_curve<<<dim3((p->K + 31) / 32, B), 256, 0, st>>>(x->kmom, B, x->key_group0, x->tab, p->mu, p->K, x->G_ws,
                                                          gcv, x->done + 1, mu_idx);
    return gx_check(p, "k_gx_curve");
}

bool gcvx_active(const hobc_plan_s* p) { return p->gcv_mode == HOBC_GCV_EXPANSION && p->gx != nullptr; }

hobc_status gcvx_prepare(hobc_plan_s* p, const void* D) {
    return fam_fourier(p->fam) ? gcvx_prepare_d<true>(p, D) : gcvx_prepare_d<false>(p, D);
}

hobc_status run_gcv_expansion(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    if (!p->gx_prepared) {                       // a view whose caller prepared the eigenvalue steps skips them
        const hobc_status s = gcvx_prepare(p, D);
        if (s != HOBC_OK) return s;
    }
    return fam_fourier(p->fam) ? gcvx_curves<true>(p, ghat, gcv, mu_idx) : gcvx_curves<false>(p, ghat, gcv, mu_idx);
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
        const hobc_status s = gcvx_setup(p);
        if (s != HOBC_OK) return s;
    }
    p->gcv_mode = HOBC_GCV_EXPANSION;
    return HOBC_OK;
}

int hobc_plan_gcv_mode(const hobc_plan* p) { return p ? p->gcv_mode : -1; }

double hobc_gcv_expansion_bound(const hobc_plan* p) { return (p && p->gx) ? p->gx->bound : -1.0; }

}  // extern "C"
