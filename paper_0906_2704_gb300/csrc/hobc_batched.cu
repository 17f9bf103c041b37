// Batched deblurring of many 2D problems of uneven sizes, each with its own
// symmetric PSF and boundary-condition degree (1: SINE, 2: COSINE,
// 3: SINE_CUBIC), in one CUDA-graph launch.
//
// The batch plan builds the transform tables once per distinct (family, n),
// lays the problems out back to back, and turns every pass of the method into
// a host-built work list: one entry per (problem, block of lines) for the line
// transforms, per (problem, chunk) for the GCV scan, per (problem, column) for
// the eigenvalues.  One kernel launch per pass and family walks its list; a
// CTA reads its entry, takes that problem's axis tables, and runs the same
// device code as the single-geometry plan (pair_analysis_body,
// pair_synthesis_body, gcv_partials_body).  Every line kernel runs 256-thread
// CTAs: an FFT of length M uses tpg threads per line pair (M/16 for M >= 256,
// M/8 below), so a CTA holds 256/tpg groups.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "hobc_internal.h"
#include "hobc_gcvx.cuh"
#include "hobc_kernels.cuh"

namespace hobc {

struct LineWork {           // one CTA of a line pass
    int item, axis, r0, nlines;
    long long in_off, out_off;
    int in_rs, in_cs, out_rs, out_cs;
    int axis_o;             // the other axis (filter smoothing)
};

struct ItemDev {            // per-problem geometry on the device
    int n0, n1, p0, p1, fam;
    int N0, N1;
    long long img_off, psf_off;
    long long cos0, cos1;   // cosine tables of the two axes: cos(k theta_t) at base + k n + t
};

struct GcvItem {
    GcvGeom geo;
    long long spec_off, part_off;
    int nchunks;
};

struct BatchIO {            // the caller's buffers of one call (read by the graph)
    const void* g;
    const void* psf;
    void* f;
    int* mu_idx;
    double* gcv;
};

static const int kBatchThreads = 256;

// ------------------------------------------------------------------ kernels

__global__ void kb_gcv_finalize(const GcvItem* __restrict__ gi, const double* __restrict__ partials,
                                const BatchIO* __restrict__ io, int K) {
    __shared__ double sv[256];
    __shared__ int si[256];
    const int item = blockIdx.x;
    const GcvItem g = gi[item];
    const double* p = partials + g.part_off;
    double best = INFINITY;
    int bi = 0x7fffffff;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        double num, den;
        sum_chunks(p, g.nchunks, K, j, num, den);
        const double Gv = num / (den * den);
        if (io->gcv) io->gcv[(long long)item * K + j] = Gv;
        const double key = isnan(Gv) ? INFINITY : Gv;
        if (key < best || (key == best && j < bi)) { best = key; bi = j; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            const double v2 = sv[threadIdx.x + s];
            const int i2 = si[threadIdx.x + s];
            if (v2 < sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) io->mu_idx[item] = si[0] == 0x7fffffff ? 0 : si[0];
}

// ----------------------------------------------------- persistent passes
// One launch per pass for every family: resident CTAs (the SMs times the CTAs
// that fit on one) take the work items of the pass's list in order from a
// device counter, one at a time, and run the same device code as the
// per-family kernels above on each.  The lists are sorted on the host by
// decreasing cost (FFT length, then lines), so the longest items start first
// and the short ones fill the tail.  The counters are zeroed by a memset node
// at the head of the graph.  Work items are independent within a pass, so no
// CTA waits on another.
// The work queue of a persistent pass: a CTA draws item k from the counter,
// and while it works on k its thread 0 has already drawn the next one (the
// atomic's latency hides behind the work); the hand-over's barriers also keep
// an item's shared memory from being overwritten while it is still read.
__device__ __forceinline__ int queue_first(int* counter, int& slot) {
    if (threadIdx.x == 0) slot = atomicAdd(counter, 1);
    __syncthreads();
    return slot;
}
__device__ __forceinline__ int queue_draw(int* counter) { return threadIdx.x == 0 ? atomicAdd(counter, 1) : 0; }
__device__ __forceinline__ int queue_handover(int drawn, int& slot) {
    __syncthreads();
    if (threadIdx.x == 0) slot = drawn;
    __syncthreads();
    return slot;
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
kp_analysis(const LineWork* __restrict__ work, int count, int* __restrict__ counter,
            const Axis<T>* __restrict__ axes, const T* __restrict__ in_fixed, int in_from_io,
            const BatchIO* __restrict__ io, T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int slot;
    for (int k = queue_first(counter, slot); k < count;) {
        const int drawn = queue_draw(counter);
        const LineWork w = work[k];
        const Axis<T>& ax = axes[w.axis];
        const T* in = (in_from_io ? reinterpret_cast<const T*>(io->g) : in_fixed) + w.in_off;
        if (ax.fam == FAM_S)
            pair_analysis_body<T, FAM_S>(in, 0, w.in_rs, out + w.out_off, 0, w.out_rs, w.out_cs, w.nlines, ax, 0,
                                         w.r0, smem_raw);
        else if (ax.fam == FAM_C)
            pair_analysis_body<T, FAM_C>(in, 0, w.in_rs, out + w.out_off, 0, w.out_rs, w.out_cs, w.nlines, ax, 0,
                                         w.r0, smem_raw);
        else
            pair_analysis_body<T, FAM_S3>(in, 0, w.in_rs, out + w.out_off, 0, w.out_rs, w.out_cs, w.nlines, ax, 0,
                                          w.r0, smem_raw);
        k = queue_handover(drawn, slot);
    }
}

template <typename T, int FMODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
kp_synthesis(const LineWork* __restrict__ work, int count, int* __restrict__ counter,
             const Axis<T>* __restrict__ axes, const T* __restrict__ in, T* __restrict__ out_fixed, int out_to_io,
             const BatchIO* __restrict__ io, const T* __restrict__ D, FilterDesc fd0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int slot;
    for (int k = queue_first(counter, slot); k < count;) {
        const int drawn = queue_draw(counter);
        const LineWork w = work[k];
        const Axis<T>& ax = axes[w.axis];
        FilterDesc fd = fd0;
        if (FMODE == 2) {
            const Axis<T>& ao = axes[w.axis_o];
            fd.D = D + w.in_off;             // eigenvalues share the spectrum layout
            fd.d_psf_stride = 0;
            fd.psf_per = 0;
            fd.mu_idx = io->mu_idx + w.item;
            fd.o_fam = ao.fam; fd.o_n = ao.n; fd.o_N = ao.N; fd.o_W = ao.W;
        }
        T* out = (out_to_io ? reinterpret_cast<T*>(io->f) : out_fixed) + w.out_off;
        if (ax.fam == FAM_S)
            pair_synthesis_body<T, FAM_S, FMODE>(in + w.in_off, 0, w.in_rs, w.in_cs, out, 0, w.out_rs, w.nlines, ax,
                                                 fd, 0, w.r0, smem_raw);
        else if (ax.fam == FAM_C)
            pair_synthesis_body<T, FAM_C, FMODE>(in + w.in_off, 0, w.in_rs, w.in_cs, out, 0, w.out_rs, w.nlines, ax,
                                                 fd, 0, w.r0, smem_raw);
        else
            pair_synthesis_body<T, FAM_S3, FMODE>(in + w.in_off, 0, w.in_rs, w.in_cs, out, 0, w.out_rs, w.nlines,
                                                  ax, fd, 0, w.r0, smem_raw);
        k = queue_handover(drawn, slot);
    }
}

// Eigenvalues of a symmetric PSF on the real families: d = sum h cos(j0 th0) cos(j1 th1)
// (Eq. (eq:symbol) at -theta, Sec. 6): partial sums over j1 for the column,
// then the sum over j0 for every entry, tap offsets +-k folded; the cosines
// cos(k theta_t) come from per-axis tables built on the host with the
// argument reduced exactly.  One work item per (problem, kEigCols columns):
// the cosine of an entry t0 is loaded once for all the item's columns.
// The partial sums are FP64.  The sums over j0 are FP64 in FP64 batches; in
// FP32 batches they are compensated dot products in float-float arithmetic
// (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005: exact
// products by FMA, error-free TwoSum of the running sum, the errors summed
// apart) of the operands split into float pairs hi + lo, within about 2^-45 of
// sum |terms| -- FP64 runs at 1/64 of the FP32 rate on this GPU, and these
// sums are n0 n1 p0 / 2 products per problem.
static const int kEigCols = 8;

template <typename T>
__global__ void __launch_bounds__(256)
kp_eig(const int2* __restrict__ work, int count, int* __restrict__ counter, const ItemDev* __restrict__ items,
       const BatchIO* __restrict__ io, const double* __restrict__ costab, const float2* __restrict__ costab2,
       T* __restrict__ D) {
    __shared__ double P[kEigCols][64];
    __shared__ double A[kEigCols][32];          // FP64 batches: A_q = P_{m0+q} + P_{m0-q}, A_0 = P_{m0}
    __shared__ float2 Af[32][kEigCols];         // FP32 batches: A_q as (hi, lo)
    __shared__ int slot;
    for (int k = queue_first(counter, slot); k < count;) {
        const int drawn = queue_draw(counter);
        const int2 w = work[k];
        const ItemDev it = items[w.x];
        const int c0 = w.y, nc = min(kEigCols, it.n1 - c0);
        const T* h = reinterpret_cast<const T*>(io->psf) + it.psf_off;
        const int m0 = it.p0 / 2, m1 = it.p1 / 2;
        for (int e = threadIdx.x; e < nc * it.p0; e += blockDim.x) {
            const int cc = e / it.p0, j0 = e - cc * it.p0;
            const double* c1t = costab + it.cos1 + c0 + cc;
            const T* hr = h + j0 * it.p1;
            double acc = (double)hr[m1];
            for (int q = 1; q <= m1; ++q) acc += ((double)hr[m1 + q] + (double)hr[m1 - q]) * c1t[(long long)q * it.n1];
            P[cc][j0] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nc * (m0 + 1); e += blockDim.x) {
            const int cc = e / (m0 + 1), q = e - cc * (m0 + 1);
            const double v = q == 0 ? P[cc][m0] : P[cc][m0 + q] + P[cc][m0 - q];
            if constexpr (sizeof(T) == 8) {
                A[cc][q] = v;
            } else {
                const float hi = (float)v;
                Af[q][cc] = make_float2(hi, (float)(v - (double)hi));
            }
        }
        __syncthreads();
        T* o = D + it.img_off + (long long)c0 * it.n0;
        for (int t0 = threadIdx.x; t0 < it.n0; t0 += blockDim.x) {
            if constexpr (sizeof(T) == 8) {
                const double* c0t = costab + it.cos0 + t0;
                double acc[kEigCols];
#pragma unroll
                for (int cc = 0; cc < kEigCols; ++cc) acc[cc] = A[cc][0];
                for (int q = 1; q <= m0; ++q) {
                    const double cq = c0t[(long long)q * it.n0];
#pragma unroll
                    for (int cc = 0; cc < kEigCols; ++cc) acc[cc] += A[cc][q] * cq;
                }
#pragma unroll
                for (int cc = 0; cc < kEigCols; ++cc)
                    if (cc < nc) o[(long long)cc * it.n0 + t0] = (T)acc[cc];
            } else {
                const float2* c0t = costab2 + it.cos0 + t0;
                float s[kEigCols], r[kEigCols];
#pragma unroll
                for (int cc = 0; cc < kEigCols; ++cc) { s[cc] = Af[0][cc].x; r[cc] = Af[0][cc].y; }
                for (int q = 1; q <= m0; ++q) {
                    const float2 cq = c0t[(long long)q * it.n0];
#pragma unroll
                    for (int cc = 0; cc < kEigCols; ++cc) {
                        const float2 a = Af[q][cc];
                        // the _rn intrinsics keep the compiler from fusing these into FMAs
                        const float p = __fmul_rn(a.x, cq.x);
                        const float pe = __fmaf_rn(a.x, cq.x, -p);           // a.x cq.x = p + pe exactly
                        const float sn = __fadd_rn(s[cc], p);                // TwoSum: s + p = sn + se exactly
                        const float bv = __fsub_rn(sn, s[cc]);
                        const float se = __fadd_rn(__fsub_rn(s[cc], __fsub_rn(sn, bv)), __fsub_rn(p, bv));
                        s[cc] = sn;
                        r[cc] += se + pe + __fmaf_rn(a.x, cq.y, a.y * cq.x);
                    }
                }
#pragma unroll
                for (int cc = 0; cc < kEigCols; ++cc)
                    if (cc < nc) o[(long long)cc * it.n0 + t0] = s[cc] + r[cc];
            }
        }
        k = queue_handover(drawn, slot);
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
kp_gcv(const int2* __restrict__ work, int count, int* __restrict__ counter, const GcvItem* __restrict__ gi,
       const T* __restrict__ G, const T* __restrict__ D, const T* __restrict__ muT, double* __restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int slot;
    for (int k = queue_first(counter, slot); k < count;) {
        const int drawn = queue_draw(counter);
        const int2 w = work[k];
        const GcvItem g = gi[w.x];
        gcv_partials_body<T, false>(G + g.spec_off, D + g.spec_off, muT, g.geo, (long long)w.y * g.geo.chunk,
                                    partials + g.part_off + (long long)w.y * 2 * g.geo.K, smem_raw);
        k = queue_handover(drawn, slot);
    }
}

// ------------------------------------------- GCV curve by bin expansion
// The batch form of the plans' expansion (hobc_gcvx.cu): every problem has its
// own eigenvalues, so the entries are grouped by key within chunks of
// kGxBChunk entries of one problem instead of by a global sort.  A work item
// (problem, chunk) classifies its entries (eight per thread, kept in registers),
// sorts them by key into shared memory (stable: per-warp counts over entry
// order, then ranks among equal keys), and writes, for every key present, the 8
// numerator and 8 denominator moments of its entries into the key's slot of the
// chunk's record, with a bit of the chunk's presence mask.  Each thread sums
// eight consecutive sorted entries run by run; a run that crosses threads is
// joined by a segmented scan over the threads (a fixed shuffle tree within a
// warp, the warps in order), so every sum has a fixed order.  A problem's curve
// then adds its chunks' moments key by key in chunk order (float-float) and
// evaluates G on the grid.
static const int kGxBChunk = 2048;
static const int kGxBPer = kGxBChunk / 256;          // entries per thread
static const int kGxLamN = 1024;                     // |s|^2 tables: positions along axis 0,
static const int kGxLamRows = 64;                    // rows of one chunk
static const int kGxMaskW = (kGxKeys + 31) / 32;     // presence mask words per chunk

struct __align__(16) GxRec {     // one key's moments within one chunk
    float E[kGxP];          // sum e u^p, e = w |ghat|^2 (w/a^2 above a_hi)
    float W[kGxP];          // sum w u^p (w/a above a_hi)
};

// One key's place in a chunk's key-sorted order (run: the entries before it):
// its start and count, and its entries' start in each of the eight warps'
// slices (in warp order).
__device__ __forceinline__ void gx_place_key(int key, int tot, int run, int (*wc)[kGxKeys], int* kstart, int* kcount) {
    kstart[key] = run;
    kcount[key] = tot;
    int r = run;
#pragma unroll
    for (int w2 = 0; w2 < 8; ++w2) {
        const int t = wc[w2][key];
        wc[w2][key] = r;
        r += t;
    }
}

__device__ __forceinline__ void gx_put_rec(GxRec* rec, long long at, const float2* c) {
    float4* o = reinterpret_cast<float4*>(rec + at);
    o[0] = make_float4(c[0].x, c[1].x, c[2].x, c[3].x);
    o[1] = make_float4(c[4].x, c[5].x, c[6].x, c[7].x);
    o[2] = make_float4(c[0].y, c[1].y, c[2].y, c[3].y);
    o[3] = make_float4(c[4].y, c[5].y, c[6].y, c[7].y);
}

// Work items in a fixed round robin over the CTAs (chunks cost the same, but
// for the last of each problem); the sums below are (E_p, W_p) pairs, added and
// scaled two at a time.
template <typename T>
__global__ void __launch_bounds__(256, 3)
kp_gcvx(const int2* __restrict__ work, int count, const GcvItem* __restrict__ gi, const int* __restrict__ chunk0,
        const T* __restrict__ G, const T* __restrict__ D, const GxTab* __restrict__ tab,
        unsigned* __restrict__ rec_mask, GxRec* __restrict__ rec) {
    __shared__ __align__(16) float su[kGxBChunk], se[kGxBChunk], sd[kGxBChunk];   // key-sorted entries
    __shared__ __align__(16) short sk[kGxBChunk];
    __shared__ int wc[8][kGxKeys];
    __shared__ int kstart[kGxKeys], kcount[kGxKeys];
    __shared__ int wsum[8];
    __shared__ float2 wagg[8][kGxP], wcar[8][kGxP];
    __shared__ int wflag[8];
    __shared__ float lam0[kGxLamN], lam1[kGxLamRows];
    __shared__ GxTab stab;
    __shared__ int ntot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    for (int j = threadIdx.x; j < (int)(sizeof(GxTab) / 4); j += blockDim.x)
        reinterpret_cast<float*>(&stab)[j] = reinterpret_cast<const float*>(tab)[j];
    for (int k = blockIdx.x; k < count; k += gridDim.x) {
        const int2 w = work[k];
        const GcvItem g = gi[w.x];
        const long long e0 = (long long)w.y * kGxBChunk;
        const int cnt = (int)min((long long)kGxBChunk, g.geo.S - e0);
        const T* Gp = G + g.spec_off;
        const T* Dp = D + g.spec_off;
        float dv[kGxBPer], gv[kGxBPer];
#pragma unroll
        for (int it = 0; it < kGxBPer; ++it) {
            const int i = warp * (kGxBChunk / 8) + it * 32 + lane;
            dv[it] = i < cnt ? (float)Dp[e0 + i] : 0.f;
            gv[it] = i < cnt ? (float)Gp[e0 + i] : 0.f;
        }
        for (int j = threadIdx.x; j < 8 * kGxKeys; j += blockDim.x) (&wc[0][0])[j] = 0;
        // |s|^2 by tables of the chunk's two Laplacian factors (the sums lap_s2 forms,
        // the same operations): one per position along axis 0, one per row in the chunk
        const GcvGeom& geo = g.geo;
        const int c_lo = (int)(e0 / geo.n0);
        const bool tabled = geo.lap && geo.ndim == 2 && geo.n0 <= kGxLamN &&
                            (cnt + geo.n0 - 1) / geo.n0 + 1 <= kGxLamRows;
        if (tabled) {
            for (int t0 = threadIdx.x; t0 < geo.n0; t0 += blockDim.x)
                lam0[t0] = lap_eig<float>(theta_over_pi<float>(geo.fam, geo.n0, geo.N0, t0));
            const int rows = (int)((e0 + cnt - 1) / geo.n0) - c_lo + 1;
            for (int r = threadIdx.x; r < rows; r += blockDim.x)
                lam1[r] = lap_eig<float>(
                    theta_over_pi<float>(geo.fam, geo.n1, geo.N1, stored_to_t(geo.fam, geo.n1, geo.W1, c_lo + r)));
        }
        // the row of offset e from row c_lo: (e + 1/2)/n0 is at least 1/(2 n0) from an
        // integer and below 2 + 2048/n0, so its FP32 product with 1/n0 truncates exactly
        const float inv_n0 = 1.f / (float)geo.n0;
        const int t_lo = (int)(e0 - (long long)c_lo * geo.n0);
        __syncthreads();
        // the entries of warp w: [256 w, 256 (w + 1)), in steps of 32; key, coordinate and
        // the two terms (real families: weight 1); key -1 for entries outside the sums
        int key[kGxBPer];
        float uu[kGxBPer], vn[kGxBPer], vd[kGxBPer];
        unsigned peers[kGxBPer];
#pragma unroll
        for (int it = 0; it < kGxBPer; ++it) {
            const int i = warp * (kGxBChunk / 8) + it * 32 + lane;
            key[it] = -1;
            uu[it] = 0.f; vn[it] = 0.f; vd[it] = 0.f;
            if (i < cnt) {
                float s2;
                if (tabled) {
                    const int e = t_lo + i;
                    const int r = (int)(((float)e + 0.5f) * inv_n0);
                    const float sv = lam1[r] + lam0[e - r * geo.n0];
                    s2 = sv * sv;
                } else {
                    int c;
                    s2 = (float)lap_s2<T>(geo, e0 + i, c);
                }
                if (s2 > 0.f) {
                    const float a = fminf(__fdividef(dv[it] * dv[it], s2), a_cap<float>());
                    key[it] = gx_classify(a, 1.f, &stab, uu[it], vn[it], vd[it]);
                    vn[it] *= gv[it] * gv[it];
                }
            }
        }
        // stable counting sort: counts per warp and key, in entry order
#pragma unroll
        for (int it = 0; it < kGxBPer; ++it) {
            peers[it] = __match_any_sync(0xffffffffu, key[it]);
            if (key[it] >= 0 && lane == __ffs(peers[it]) - 1) wc[warp][key[it]] += __popc(peers[it]);
            __syncwarp();
        }
        __syncthreads();
        const long long chunk = chunk0[w.x] + w.y;
        {
            // key starts in key order: one block-wide exclusive scan of the counts over
            // keys 0..255 (a key per thread), keys 256 and 257 after them; then each key's
            // warp prefixes, and the presence mask
            const int kk = threadIdx.x;
            int tk = 0;
#pragma unroll
            for (int w2 = 0; w2 < 8; ++w2) tk += wc[w2][kk];
            int tk2 = 0, t256 = 0;
            if (threadIdx.x < kGxKeys - 256) {
#pragma unroll
                for (int w2 = 0; w2 < 8; ++w2) {
                    t256 += wc[w2][256];
                    tk2 += wc[w2][256 + threadIdx.x];
                }
            }
            const unsigned present = __ballot_sync(0xffffffffu, tk > 0);
            if (lane == 0) rec_mask[chunk * kGxMaskW + warp] = present;
            int inc = tk;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc += y;
            }
            if (lane == 31) wsum[warp] = inc;
            __syncthreads();
            int base = 0, all = 0;
#pragma unroll
            for (int w2 = 0; w2 < 8; ++w2) {
                if (w2 < warp) base += wsum[w2];
                all += wsum[w2];
            }
            gx_place_key(kk, tk, base + inc - tk, wc, kstart, kcount);
            if (threadIdx.x < kGxKeys - 256) {
                gx_place_key(256 + threadIdx.x, tk2, all + (threadIdx.x == 1 ? t256 : 0), wc, kstart, kcount);
                if (threadIdx.x == 1) {
                    ntot = all + t256 + tk2;
                    rec_mask[chunk * kGxMaskW + 8] = (t256 > 0 ? 1u : 0u) | (tk2 > 0 ? 2u : 0u);
                }
            }
        }
        __syncthreads();
        // scatter into key order: the warp's start for the key, then the rank among equal keys
#pragma unroll
        for (int it = 0; it < kGxBPer; ++it) {
            if (key[it] >= 0) {
                const int pos = wc[warp][key[it]] + __popc(peers[it] & lt);
                su[pos] = uu[it]; se[pos] = vn[it]; sd[pos] = vd[it]; sk[pos] = (short)key[it];
            }
            __syncwarp();
            if (key[it] >= 0 && lane == __ffs(peers[it]) - 1) wc[warp][key[it]] += __popc(peers[it]);
            __syncwarp();
        }
        __syncthreads();
        // each thread: sorted entries [8 t, 8 t + 8), run by run.  A run inside the
        // thread is written at once; one that began in an earlier thread and ends here
        // (the thread owns it) waits for the carry; one that goes on past the thread is
        // its contribution X to the segmented scan (flag F: a run begins here)
        const long long rbase = chunk * kGxKeys;
        const int p0 = threadIdx.x * kGxBPer, n = ntot;
        float2 c2[kGxP], o2[kGxP];
#pragma unroll
        for (int p = 0; p < kGxP; ++p) { c2[p] = make_float2(0.f, 0.f); o2[p] = make_float2(0.f, 0.f); }
        int curk = -1, okey = -1;
        if (p0 < n) {
            const float4 u4[2] = {reinterpret_cast<const float4*>(su + p0)[0],
                                  reinterpret_cast<const float4*>(su + p0)[1]};
            const float4 e4[2] = {reinterpret_cast<const float4*>(se + p0)[0],
                                  reinterpret_cast<const float4*>(se + p0)[1]};
            const float4 d4[2] = {reinterpret_cast<const float4*>(sd + p0)[0],
                                  reinterpret_cast<const float4*>(sd + p0)[1]};
            const short* kp = sk + p0;
            const float* ua = reinterpret_cast<const float*>(u4);
            const float* ea = reinterpret_cast<const float*>(e4);
            const float* da = reinterpret_cast<const float*>(d4);
#pragma unroll
            for (int j = 0; j < kGxBPer; ++j) {
                if (p0 + j < n) {
                    const int kj = kp[j];
                    if (kj != curk) {
                        if (curk >= 0) {                // the run of curk ends at p0 + j - 1
                            if (kstart[curk] < p0) {
                                okey = curk;
#pragma unroll
                                for (int p = 0; p < kGxP; ++p) o2[p] = c2[p];
                            } else {
                                gx_put_rec(rec, rbase + curk, c2);
                            }
#pragma unroll
                            for (int p = 0; p < kGxP; ++p) c2[p] = make_float2(0.f, 0.f);
                        }
                        curk = kj;
                    }
                    float2 t2 = make_float2(ea[j], da[j]);
                    const float2 u2 = make_float2(ua[j], ua[j]);
#pragma unroll
                    for (int p = 0; p < kGxP; ++p) {
                        c2[p] = __fadd2_rn(c2[p], t2);
                        t2 = __fmul2_rn(t2, u2);
                    }
                }
            }
        }
        int F = 1;
        if (curk >= 0) {
            const bool starts = kstart[curk] >= p0, ends = kstart[curk] + kcount[curk] <= p0 + kGxBPer;
            if (ends) {
                if (starts) {
                    gx_put_rec(rec, rbase + curk, c2);
                } else {
                    okey = curk;
#pragma unroll
                    for (int p = 0; p < kGxP; ++p) o2[p] = c2[p];
                }
#pragma unroll
                for (int p = 0; p < kGxP; ++p) c2[p] = make_float2(0.f, 0.f);
            } else {
                F = starts ? 1 : 0;
            }
        }
        // segmented inclusive scan of (X, F) over the threads: within the warp...
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int yF = __shfl_up_sync(0xffffffffu, F, off);
#pragma unroll
            for (int p = 0; p < kGxP; ++p) {
                float2 y;
                y.x = __shfl_up_sync(0xffffffffu, c2[p].x, off);
                y.y = __shfl_up_sync(0xffffffffu, c2[p].y, off);
                if (lane >= off && !F) c2[p] = __fadd2_rn(y, c2[p]);
            }
            if (lane >= off) F |= yF;
        }
        if (lane == 31) {
#pragma unroll
            for (int p = 0; p < kGxP; ++p) wagg[warp][p] = c2[p];
            wflag[warp] = F;
        }
        __syncthreads();
        // ...then the warps in order: the carry into each warp (a thread per warp and pair)
        if (threadIdx.x < 8 * kGxP) {
            const int wv = threadIdx.x / kGxP, q = threadIdx.x % kGxP;
            float2 C = make_float2(0.f, 0.f);
            for (int w2 = 0; w2 < wv; ++w2) C = wflag[w2] ? wagg[w2][q] : __fadd2_rn(C, wagg[w2][q]);
            wcar[wv][q] = C;
        }
        __syncthreads();
        if (!F) {
#pragma unroll
            for (int p = 0; p < kGxP; ++p) c2[p] = __fadd2_rn(wcar[warp][p], c2[p]);
        }
        // the owner of a run that began earlier: the previous thread's scanned sums + its own
#pragma unroll
        for (int p = 0; p < kGxP; ++p) {
            float2 y;
            y.x = __shfl_up_sync(0xffffffffu, c2[p].x, 1);
            y.y = __shfl_up_sync(0xffffffffu, c2[p].y, 1);
            o2[p] = __fadd2_rn(lane == 0 ? wcar[warp][p] : y, o2[p]);
        }
        if (okey >= 0) gx_put_rec(rec, rbase + okey, o2);
        __syncthreads();                // the shared arrays are reused by the next work item
    }
}

// The curve of every problem: its chunks' moments added key by key in chunk
// order (float-float; a thread per key and moment, the chunks whose mask has
// the key), G(mu_j) for every grid value (Horner in FP32 per key, float-float
// over the keys, two key halves per grid value added in order), and the first
// minimum (NaN never wins).  One CTA per problem.
__global__ void __launch_bounds__(256)
kb_gxcurve(const int* __restrict__ chunk0, const unsigned* __restrict__ rec_mask, const GxRec* __restrict__ rec,
           const GxTab* __restrict__ tab, const double* __restrict__ mu, int K, const BatchIO* __restrict__ io) {
    __shared__ float Ms[kGxKeys][2 * kGxP];       // E_p (p + 1), then W_p
    __shared__ float red[4][2][128];
    __shared__ double sv[256];
    __shared__ int si[256];
    const int item = blockIdx.x;
    const long long c0 = chunk0[item];
    const int nch = chunk0[item + 1] - chunk0[item];
    for (int q = threadIdx.x; q < kGxKeys * 2 * kGxP; q += blockDim.x) {
        const int key = q / (2 * kGxP), comp = q % (2 * kGxP);
        const unsigned bit = 1u << (key & 31);
        const unsigned* mk = rec_mask + c0 * kGxMaskW + (key >> 5);
        const float* rv = reinterpret_cast<const float*>(rec + c0 * kGxKeys + key) + comp;
        float hi = 0.f, lo = 0.f;
#pragma unroll 4
        for (int c = 0; c < nch; ++c)
            if (__ldg(mk + (long long)c * kGxMaskW) & bit) two_sum_acc(hi, lo, __ldg(rv + (long long)c * kGxKeys * 2 * kGxP));
        Ms[key][comp] = comp < kGxP ? (hi + lo) * (float)(comp + 1) : hi + lo;
    }
    __syncthreads();
    double best = INFINITY;
    int bi = 0x7fffffff;
    const int half = threadIdx.x >> 7, jl = threadIdx.x & 127;   // two key halves per grid value
    for (int jb = 0; jb < K; jb += 128) {
        const int j = jb + jl;
        const float m = j < K ? (float)mu[j] : 1.f;
        float nh = 0, nl = 0, dh = 0, dl = 0;
        for (int key = half; key < kGxKeys; key += 2) {
            float x, sn_, sd_;
            gx_key_terms(key, m, tab, x, sn_, sd_);
            float hn = Ms[key][kGxP - 1], hd = Ms[key][2 * kGxP - 1];
#pragma unroll
            for (int p = kGxP - 2; p >= 0; --p) {
                hn = fmaf(hn, x, Ms[key][p]);
                hd = fmaf(hd, x, Ms[key][kGxP + p]);
            }
            two_sum_acc(nh, nl, hn * sn_);
            two_sum_acc(dh, dl, hd * sd_);
        }
        red[0][half][jl] = nh; red[1][half][jl] = nl; red[2][half][jl] = dh; red[3][half][jl] = dl;
        __syncthreads();
        if (half == 0 && j < K) {
            float ah = red[0][0][jl], al = red[1][0][jl], bh = red[2][0][jl], bl = red[3][0][jl];
            two_sum_acc(ah, al, red[0][1][jl]);
            al += red[1][1][jl];
            two_sum_acc(bh, bl, red[2][1][jl]);
            bl += red[3][1][jl];
            const double den = (double)bh + (double)bl;
            const double Gv = ((double)ah + (double)al) / (den * den);
            if (io->gcv) io->gcv[(long long)item * K + j] = Gv;
            const double key = isnan(Gv) ? INFINITY : Gv;
            if (key < best || (key == best && j < bi)) { best = key; bi = j; }
        }
        __syncthreads();
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            const double v2 = sv[threadIdx.x + s];
            const int i2 = si[threadIdx.x + s];
            if (v2 < sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) io->mu_idx[item] = si[0] == 0x7fffffff ? 0 : si[0];
}

}  // namespace hobc

using namespace hobc;

// ----------------------------------------------------------------- the plan

struct PassList {           // one launch: a family's work list for one pass
    int fam;
    LineWork* dev;
    int count;
    size_t smem;
};

struct hobc_batch_s {
    hobc_batch_desc desc;
    int count, K, prec;
    size_t esz;
    cudaStream_t stream;
    std::vector<hobc_batch_item> items;
    std::vector<size_t> img_off, psf_off;
    std::vector<AxisHost> axes_host;
    void* axes_dev;
    ItemDev* items_dev;
    GcvItem* gcv_items_dev;
    int2* gcv_work;
    int gcv_count;
    int2* eig_work;
    int eig_count;
    PassList pass[4];        // row analysis, column analysis, column synthesis (+ filter), row synthesis
    int* counters;           // [6] work counters of the persistent passes (eig, 4 line passes, gcv)
    int grid[6];             // resident CTAs of each persistent pass
    std::vector<hobc_fft_schedule> schedule;   // the radix of every (degree, FFT length) the caller chose
    double* mu;
    void* muT;
    void *R, *G, *D;
    double* partials;
    int* mu_idx_ws;
    double* gcv_ws;
    BatchIO* io_dev;
    double* costab;          // per-axis tables cos(k theta_t), k <= the largest PSF half-width
    float2* costab2;         // the same split into float pairs hi + lo (FP32 batches)
    int gcv_mode;            // HOBC_GCV_DIRECT / HOBC_GCV_EXPANSION (FP32 batches)
    GxTab* gxtab;            // the expansion's bin geometry
    int2* gx_work;           // (problem, chunk of kGxBChunk entries), costliest first
    int gx_count;
    int* gx_chunk0;          // [count + 1] first chunk of each problem
    unsigned* rec_mask;      // [chunks][kGxMaskW] keys present in each chunk
    GxRec* rec;              // [chunks][keys] their moments (slots of absent keys unwritten)
    int gx_grid;
    double gx_bound;
    cudaGraphExec_t graph;
    int launches;
};

namespace {

int family_of(int degree) {
    return degree == 1 ? FAM_S : degree == 2 ? FAM_C : degree == 3 ? FAM_S3 : -1;
}

template <typename T>
hobc_status launch_all(hobc_batch_s* b) {
    cudaStream_t st = b->stream;
    const BatchIO* io = b->io_dev;
    const Axis<T>* axes = reinterpret_cast<const Axis<T>*>(b->axes_dev);
    T* R = reinterpret_cast<T*>(b->R);
    T* G = reinterpret_cast<T*>(b->G);
    T* D = reinterpret_cast<T*>(b->D);
    int launches = 0;
    cudaError_t e = cudaMemsetAsync(b->counters, 0, 6 * sizeof(int), st);
    if (e != cudaSuccess) { set_last_error("hobc_deblur_batched", e); return HOBC_ERR_CUDA; }
    int* ctr = b->counters;
    if (b->eig_count) {
        kp_eig<T><<<b->grid[0], 256, 0, st>>>(b->eig_work, b->eig_count, ctr + 0, b->items_dev, io, b->costab, b->costab2,
                                               D);
        ++launches;
    }
    const PassList* P = b->pass;
    if (P[0].count) {
        kp_analysis<T><<<b->grid[1], kBatchThreads, P[0].smem, st>>>(P[0].dev, P[0].count, ctr + 1, axes, nullptr, 1,
                                                                      io, R);
        ++launches;
    }
    if (P[1].count) {
        kp_analysis<T><<<b->grid[2], kBatchThreads, P[1].smem, st>>>(P[1].dev, P[1].count, ctr + 2, axes, R, 0, io,
                                                                      G);
        ++launches;
    }
    if (sizeof(T) == 4 && b->gcv_mode == HOBC_GCV_EXPANSION) {
        kp_gcvx<T><<<b->gx_grid, 256, 0, st>>>(b->gx_work, b->gx_count, b->gcv_items_dev, b->gx_chunk0, G, D,
                                               b->gxtab, b->rec_mask, b->rec);
        kb_gxcurve<<<b->count, 256, 0, st>>>(b->gx_chunk0, b->rec_mask, b->rec, b->gxtab, b->mu, b->K,
                                             io);
    } else {
        const size_t gsmem = 4 * (size_t)gcv_chunk_for(1LL << 40, b->K, sizeof(T) == 8) * sizeof(T);
        kp_gcv<T><<<b->grid[5], 256, gsmem, st>>>(b->gcv_work, b->gcv_count, ctr + 5, b->gcv_items_dev, G, D,
                                                  reinterpret_cast<const T*>(b->muT), b->partials);
        kb_gcv_finalize<<<b->count, 256, 0, st>>>(b->gcv_items_dev, b->partials, io, b->K);
    }
    launches += 2;
    FilterDesc fd;
    memset(&fd, 0, sizeof(fd));
    fd.mu = b->mu;
    fd.K = b->K;
    fd.lap = b->desc.L == HOBC_L_LAPLACIAN;
    if (P[2].count) {
        kp_synthesis<T, 2><<<b->grid[3], kBatchThreads, P[2].smem, st>>>(P[2].dev, P[2].count, ctr + 3, axes, G, R, 0,
                                                                          io, D, fd);
        ++launches;
    }
    if (P[3].count) {
        kp_synthesis<T, 0><<<b->grid[4], kBatchThreads, P[3].smem, st>>>(P[3].dev, P[3].count, ctr + 4, axes, R,
                                                                          nullptr, 1, io, D, fd);
        ++launches;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error("hobc_deblur_batched launch", e); return HOBC_ERR_CUDA; }
    b->launches = launches;
    return HOBC_OK;
}

// Resident CTAs of a persistent kernel: the SMs times the CTAs that fit on one.
template <typename K>
int resident_ctas(K kernel, size_t smem, int work) {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, smem) != cudaSuccess || per < 1) per = 1;
    return std::max(1, std::min(work, sms * per));
}

template <typename T>
cudaError_t prepare_batched() {
    const int lim = 200 * 1024;
    cudaError_t e = cudaSuccess;
#define HOBC_BSMEM(k) if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
    HOBC_BSMEM((kp_analysis<T>));
    HOBC_BSMEM((kp_synthesis<T, 0>));
    HOBC_BSMEM((kp_synthesis<T, 2>));
    HOBC_BSMEM((kp_gcv<T>));
#undef HOBC_BSMEM
    return e;
}

template <typename T>
Axis<T> to_dev_axis(const AxisHost& a) {
    Axis<T> x;
    memset(&x, 0, sizeof(x));
    x.fam = a.fam; x.n = a.n; x.N = a.N; x.L = a.L; x.M = a.M; x.log2M = a.log2M;
    x.blue = a.blue; x.tpg = a.tpg; x.r16 = a.r16; x.Mp = group_slots(a.M); x.H = a.H; x.W = a.W;
    x.sslot = -1;                     // the persistent passes size a separate stage for every family
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

template <typename T>
void* upload(const std::vector<T>& v, cudaError_t& err) {
    void* d = nullptr;
    if (err == cudaSuccess && !v.empty()) err = cudaMalloc(&d, v.size() * sizeof(T));
    if (err == cudaSuccess && !v.empty()) err = cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return d;
}

}  // namespace

extern "C" void hobc_batch_destroy(hobc_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (AxisHost& a : b->axes_host) {
        cudaFree(a.tw); cudaFree(a.chirp); cudaFree(a.bhat); cudaFree(a.post); cudaFree(a.q); cudaFree(a.q2);
        cudaFree(a.etab);
        cudaFree(a.etab2);
    }
    for (PassList& l : b->pass) cudaFree(l.dev);
    cudaFree(b->counters);
    cudaFree(b->axes_dev); cudaFree(b->items_dev); cudaFree(b->gcv_items_dev); cudaFree(b->gcv_work);
    cudaFree(b->costab);
    cudaFree(b->costab2);
    cudaFree(b->gxtab); cudaFree(b->gx_work); cudaFree(b->gx_chunk0); cudaFree(b->rec_mask); cudaFree(b->rec);
    cudaFree(b->eig_work); cudaFree(b->mu); cudaFree(b->muT); cudaFree(b->R); cudaFree(b->G); cudaFree(b->D);
    cudaFree(b->partials); cudaFree(b->mu_idx_ws); cudaFree(b->gcv_ws); cudaFree(b->io_dev);
    delete b;
}

extern "C" hobc_status hobc_batch_create_tuned(const hobc_batch_desc* desc, const hobc_batch_item* items,
                                               const double* mu_grid_host, const hobc_fft_schedule* schedule,
                                               int schedule_len, void* cuda_stream, hobc_batch** out) {
    if (!out) return HOBC_ERR_ARG;
    *out = nullptr;
    if (!desc || !items || !mu_grid_host || schedule_len < 0 || (schedule_len > 0 && !schedule)) return HOBC_ERR_ARG;
    for (int k = 0; k < schedule_len; ++k) {
        const hobc_fft_schedule& e = schedule[k];
        if (family_of(e.bc_degree) < 0 || e.fft_length < 8 || (e.fft_length & (e.fft_length - 1)) ||
            (e.radix != 0 && e.radix != 8 && e.radix != 16))
            return HOBC_ERR_ARG;
    }
    const hobc_batch_desc d = *desc;
    if (d.count < 1 || d.n_mu < 1) return HOBC_ERR_ARG;
    if (d.prec != HOBC_FP64 && d.prec != HOBC_FP32) return HOBC_ERR_ARG;
    if (d.gcv_mode != HOBC_GCV_DIRECT && d.gcv_mode != HOBC_GCV_EXPANSION) return HOBC_ERR_ARG;
    if (d.L != HOBC_L_IDENTITY && d.L != HOBC_L_LAPLACIAN) return HOBC_ERR_ARG;
    for (int j = 0; j < d.n_mu; ++j) {
        if (!std::isfinite(mu_grid_host[j])) return HOBC_ERR_NONFINITE;
        if (!(mu_grid_host[j] > 0)) return HOBC_ERR_ARG;
        if (d.prec == HOBC_FP32 && (mu_grid_host[j] < 1e-18 || mu_grid_host[j] > 1e18)) return HOBC_ERR_ARG;
    }
    GxTab gxt;
    double gxb = 0;
    if (d.gcv_mode == HOBC_GCV_EXPANSION) {
        if (d.prec != HOBC_FP32) {
            set_last_error_text("hobc_batch_create: the GCV expansion serves FP32 batches");
            return HOBC_ERR_UNSUPPORTED;
        }
        gx_make_table(mu_grid_host, d.n_mu, gxt, &gxb);
        if (!(gxb <= 1e-8)) {
            set_last_error_text("hobc_batch_create: the mu grid spans too many decades for the GCV expansion");
            return HOBC_ERR_UNSUPPORTED;
        }
    }
    for (int i = 0; i < d.count; ++i) {
        const hobc_batch_item& it = items[i];
        const int fam = family_of(it.bc_degree);
        if (fam < 0) return HOBC_ERR_UNSUPPORTED;
        const int border = fam == FAM_S3 ? 4 : 2;
        for (int a = 0; a < 2; ++a) {
            const int nmax = fam == FAM_C ? 1024 : 512;          // FFT length M <= 2048
            if (it.n[a] < 8 || it.n[a] > nmax) return HOBC_ERR_SIZE;
            if (it.psf[a] < 1 || it.psf[a] % 2 == 0 || it.psf[a] > 63) return HOBC_ERR_SIZE;
            if (it.psf[a] > it.n[a] - border) return HOBC_ERR_SIZE;
        }
    }
    hobc_batch_s* b = new hobc_batch_s();
    b->schedule.assign(schedule, schedule + schedule_len);
    b->desc = d;
    b->count = d.count;
    b->K = d.n_mu;
    b->prec = d.prec;
    b->esz = d.prec == HOBC_FP64 ? 8 : 4;
    b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    b->items.assign(items, items + d.count);
    cudaError_t err = d.prec == HOBC_FP64 ? prepare_batched<double>() : prepare_batched<float>();

    // distinct axes and offsets
    std::map<std::pair<int, int>, int> axis_id;
    auto axis_of = [&](int fam, int n) {
        auto key = std::make_pair(fam, n);
        auto itr = axis_id.find(key);
        if (itr != axis_id.end()) return itr->second;
        // the radix the schedule gives this (degree, FFT length), else the default
        const int deg = fam == FAM_S ? 1 : fam == FAM_C ? 2 : 3;
        const int M = fft_length_of(fam, n);
        int radix = 0;
        for (const hobc_fft_schedule& e : b->schedule)
            if (e.bc_degree == deg && e.fft_length == M) radix = e.radix;
        AxisHost a;
        if (err == cudaSuccess)
            err = d.prec == HOBC_FP64 ? build_axis_host<double>(a, fam, n, 1, false, radix)
                                      : build_axis_host<float>(a, fam, n, 1, false, radix);
        b->axes_host.push_back(a);
        const int id = (int)b->axes_host.size() - 1;
        axis_id[key] = id;
        return id;
    };
    std::vector<ItemDev> idev(d.count);
    std::vector<int> ax0(d.count), ax1(d.count);
    b->img_off.assign(d.count + 1, 0);
    b->psf_off.assign(d.count + 1, 0);
    for (int i = 0; i < d.count; ++i) {
        const hobc_batch_item& it = items[i];
        const int fam = family_of(it.bc_degree);
        ax0[i] = axis_of(fam, it.n[0]);
        ax1[i] = axis_of(fam, it.n[1]);
        b->img_off[i + 1] = b->img_off[i] + (size_t)it.n[0] * it.n[1];
        b->psf_off[i + 1] = b->psf_off[i] + (size_t)it.psf[0] * it.psf[1];
        ItemDev& x = idev[i];
        x.n0 = it.n[0]; x.n1 = it.n[1]; x.p0 = it.psf[0]; x.p1 = it.psf[1]; x.fam = fam;
        x.N0 = fam == FAM_S3 ? x.n0 - 4 : x.n0 - 2;
        x.N1 = fam == FAM_S3 ? x.n1 - 4 : x.n1 - 2;
        x.img_off = (long long)b->img_off[i];
        x.psf_off = (long long)b->psf_off[i];
    }
    // cosine tables of every distinct axis: cos(k theta_t) for k <= the largest half-width
    {
        int kc = 1;
        for (int i = 0; i < d.count; ++i) kc = std::max(kc, std::max(items[i].psf[0], items[i].psf[1]) / 2 + 1);
        std::vector<long long> base(b->axes_host.size());
        long long total_cos = 0;
        for (size_t a = 0; a < b->axes_host.size(); ++a) {
            base[a] = total_cos;
            total_cos += (long long)kc * b->axes_host[a].n;
        }
        std::vector<double> tab((size_t)total_cos);
        for (size_t a = 0; a < b->axes_host.size(); ++a) {
            const AxisHost& ah = b->axes_host[a];
            for (int t = 0; t < ah.n; ++t) {
                long long num, den;
                theta_frac(ah.fam, ah.n, t, num, den);
                for (int k = 0; k < kc; ++k) tab[(size_t)(base[a] + (long long)k * ah.n + t)] = expm_ipi(k * num, den).real();
            }
        }
        for (int i = 0; i < d.count; ++i) {
            idev[i].cos0 = base[ax0[i]];
            idev[i].cos1 = base[ax1[i]];
        }
        b->costab = reinterpret_cast<double*>(upload(tab, err));
        std::vector<float2> tab2(tab.size());
        for (size_t k = 0; k < tab.size(); ++k) {
            const float hi = (float)tab[k];
            tab2[k] = make_float2(hi, (float)(tab[k] - (double)hi));
        }
        b->costab2 = reinterpret_cast<float2*>(upload(tab2, err));
    }
    if (err == cudaSuccess) {
        if (d.prec == HOBC_FP64) {
            std::vector<Axis<double>> v;
            for (auto& a : b->axes_host) v.push_back(to_dev_axis<double>(a));
            b->axes_dev = upload(v, err);
        } else {
            std::vector<Axis<float>> v;
            for (auto& a : b->axes_host) v.push_back(to_dev_axis<float>(a));
            b->axes_dev = upload(v, err);
        }
    }
    b->items_dev = reinterpret_cast<ItemDev*>(upload(idev, err));

    // line work lists of the four passes, every family in one list: a work item
    // covers 2G lines of a problem, G = 256/tpg; items sorted by decreasing FFT
    // length, then decreasing line count, so the costliest start first
    const size_t csz = 2 * b->esz;
    auto build_pass = [&](PassList& l, int pass) {
        std::vector<LineWork> w;
        std::vector<int> cost;
        size_t smem = 0;
        for (int i = 0; i < d.count; ++i) {
            const int n0 = idev[i].n0, n1 = idev[i].n1;
            const bool rows = pass == 0 || pass == 3;         // row passes run along axis 1
            const int ax = rows ? ax1[i] : ax0[i];
            const AxisHost& a = b->axes_host[ax];
            const int G = kBatchThreads / a.tpg;
            const int nl = rows ? n0 : n1;
            smem = std::max(smem, (size_t)G * group_slots(a.M) * csz + (size_t)2 * G * a.W * b->esz);
            for (int r0 = 0; r0 < nl; r0 += 2 * G) {
                LineWork e;
                memset(&e, 0, sizeof(e));
                e.item = i; e.axis = ax; e.r0 = r0; e.nlines = nl;
                e.in_off = e.out_off = idev[i].img_off;
                e.axis_o = ax1[i];
                if (pass == 0) { e.in_rs = n1; e.out_rs = 1; e.out_cs = n0; }            // rows -> R[c][r]
                else if (pass == 1) { e.in_rs = n0; e.out_rs = n0; e.out_cs = 1; }       // R columns -> G
                else if (pass == 2) { e.in_rs = n0; e.in_cs = 1; e.out_rs = n0; }        // G -> R (filter)
                else { e.in_rs = 1; e.in_cs = n0; e.out_rs = n1; }                        // R -> f rows
                w.push_back(e);
                cost.push_back(a.M * std::min(2 * G, nl - r0));
            }
        }
        std::vector<int> order(w.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
        // equal costs grouped by family: CTAs that run at the same time then mostly
        // run the same family's code
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            if (cost[x] != cost[y]) return cost[x] > cost[y];
            return b->axes_host[w[x].axis].fam < b->axes_host[w[y].axis].fam;
        });
        std::vector<LineWork> sorted(w.size());
        for (size_t k = 0; k < order.size(); ++k) sorted[k] = w[order[k]];
        l.fam = -1;
        l.count = (int)sorted.size();
        l.smem = smem;
        l.dev = reinterpret_cast<LineWork*>(upload(sorted, err));
    };
    for (int ps = 0; ps < 4; ++ps) build_pass(b->pass[ps], ps);

    // GCV and eigenvalue work
    std::vector<GcvItem> gi(d.count);
    std::vector<int2> gw, ew;
    long long part = 0;
    for (int i = 0; i < d.count; ++i) {
        GcvItem& g = gi[i];
        memset(&g, 0, sizeof(g));
        const AxisHost& a0 = b->axes_host[ax0[i]];
        const AxisHost& a1 = b->axes_host[ax1[i]];
        g.geo.ndim = 2; g.geo.fam = idev[i].fam;
        g.geo.n0 = a0.n; g.geo.N0 = a0.N; g.geo.n1 = a1.n; g.geo.N1 = a1.N; g.geo.W1 = a1.W;
        g.geo.lap = d.L == HOBC_L_LAPLACIAN;
        g.geo.S = (long long)a1.W * a0.n;
        g.geo.chunk = gcv_chunk_for(g.geo.S, b->K, d.prec == HOBC_FP64);
        g.geo.K = b->K;
        g.nchunks = (int)((g.geo.S + g.geo.chunk - 1) / g.geo.chunk);
        g.spec_off = idev[i].img_off;
        g.part_off = part;
        part += (long long)g.nchunks * 2 * b->K;
        for (int c = 0; c < g.nchunks; ++c) gw.push_back(make_int2(i, c));
        for (int c = 0; c < idev[i].n1; c += kEigCols) ew.push_back(make_int2(i, c));
    }
    // costliest first: eigenvalue columns by n0 p0, GCV chunks by their size
    std::stable_sort(ew.begin(), ew.end(), [&](const int2& x, const int2& y) {
        return (long long)idev[x.x].n0 * idev[x.x].p0 > (long long)idev[y.x].n0 * idev[y.x].p0;
    });
    std::stable_sort(gw.begin(), gw.end(), [&](const int2& x, const int2& y) {
        const long long cx = std::min((long long)gi[x.x].geo.chunk, gi[x.x].geo.S - (long long)x.y * gi[x.x].geo.chunk);
        const long long cy = std::min((long long)gi[y.x].geo.chunk, gi[y.x].geo.S - (long long)y.y * gi[y.x].geo.chunk);
        return cx > cy;
    });
    b->gcv_count = (int)gw.size();
    b->eig_count = (int)ew.size();
    // the expansion's work: chunks of kGxBChunk entries of each problem, costliest first
    b->gcv_mode = d.gcv_mode;
    b->gx_bound = gxb;
    std::vector<int> gx_chunk0(d.count + 1, 0);
    std::vector<int2> gxw;
    if (d.gcv_mode == HOBC_GCV_EXPANSION) {
        for (int i = 0; i < d.count; ++i) {
            const int nch = (int)((gi[i].geo.S + kGxBChunk - 1) / kGxBChunk);
            gx_chunk0[i + 1] = gx_chunk0[i] + nch;
            for (int c = 0; c < nch; ++c) gxw.push_back(make_int2(i, c));
        }
        std::stable_sort(gxw.begin(), gxw.end(), [&](const int2& x, const int2& y) {
            return std::min((long long)kGxBChunk, gi[x.x].geo.S - (long long)x.y * kGxBChunk) >
                   std::min((long long)kGxBChunk, gi[y.x].geo.S - (long long)y.y * kGxBChunk);
        });
        b->gx_count = (int)gxw.size();
        b->gx_work = reinterpret_cast<int2*>(upload(gxw, err));
        b->gx_chunk0 = reinterpret_cast<int*>(upload(gx_chunk0, err));
        std::vector<GxTab> tv(1, gxt);
        b->gxtab = reinterpret_cast<GxTab*>(upload(tv, err));
    }
    b->gcv_items_dev = reinterpret_cast<GcvItem*>(upload(gi, err));
    b->gcv_work = reinterpret_cast<int2*>(upload(gw, err));
    b->eig_work = reinterpret_cast<int2*>(upload(ew, err));

    const size_t total = b->img_off[d.count];
    auto alloc = [&](void** p, size_t bytes) { if (err == cudaSuccess && bytes) err = cudaMalloc(p, bytes); };
    alloc(&b->R, total * b->esz);
    alloc(&b->G, total * b->esz);
    alloc(&b->D, total * b->esz);
    alloc((void**)&b->partials, (size_t)part * sizeof(double));
    alloc((void**)&b->mu_idx_ws, (size_t)d.count * sizeof(int));
    alloc((void**)&b->gcv_ws, (size_t)d.count * b->K * sizeof(double));
    alloc((void**)&b->io_dev, sizeof(BatchIO));
    alloc((void**)&b->counters, 6 * sizeof(int));
    if (d.gcv_mode == HOBC_GCV_EXPANSION) {
        const size_t nch = (size_t)gx_chunk0[d.count];
        alloc((void**)&b->rec_mask, nch * kGxMaskW * sizeof(unsigned));
        alloc((void**)&b->rec, nch * kGxKeys * sizeof(GxRec));
        if (err == cudaSuccess) b->gx_grid = resident_ctas(kp_gcvx<float>, 0, b->gx_count);
    }
    if (err == cudaSuccess) {
        const size_t gsmem = 4 * (size_t)gcv_chunk_for(1LL << 40, b->K, d.prec == HOBC_FP64) * b->esz;
        const bool f64 = d.prec == HOBC_FP64;
        b->grid[0] = f64 ? resident_ctas(kp_eig<double>, 0, b->eig_count) : resident_ctas(kp_eig<float>, 0, b->eig_count);
        b->grid[1] = f64 ? resident_ctas(kp_analysis<double>, b->pass[0].smem, b->pass[0].count)
                         : resident_ctas(kp_analysis<float>, b->pass[0].smem, b->pass[0].count);
        b->grid[2] = f64 ? resident_ctas(kp_analysis<double>, b->pass[1].smem, b->pass[1].count)
                         : resident_ctas(kp_analysis<float>, b->pass[1].smem, b->pass[1].count);
        b->grid[3] = f64 ? resident_ctas(kp_synthesis<double, 2>, b->pass[2].smem, b->pass[2].count)
                         : resident_ctas(kp_synthesis<float, 2>, b->pass[2].smem, b->pass[2].count);
        b->grid[4] = f64 ? resident_ctas(kp_synthesis<double, 0>, b->pass[3].smem, b->pass[3].count)
                         : resident_ctas(kp_synthesis<float, 0>, b->pass[3].smem, b->pass[3].count);
        b->grid[5] = f64 ? resident_ctas(kp_gcv<double>, gsmem, b->gcv_count)
                         : resident_ctas(kp_gcv<float>, gsmem, b->gcv_count);
    }
    alloc((void**)&b->mu, sizeof(double) * b->K);
    alloc(&b->muT, b->esz * b->K);
    if (err == cudaSuccess) err = cudaMemcpy(b->mu, mu_grid_host, sizeof(double) * b->K, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) {
        if (d.prec == HOBC_FP64) {
            err = cudaMemcpy(b->muT, mu_grid_host, sizeof(double) * b->K, cudaMemcpyHostToDevice);
        } else {
            std::vector<float> mf(mu_grid_host, mu_grid_host + b->K);
            err = cudaMemcpy(b->muT, mf.data(), sizeof(float) * b->K, cudaMemcpyHostToDevice);
        }
    }
    if (err != cudaSuccess) {
        set_last_error("hobc_batch_create", err);
        hobc_batch_destroy(b);
        return HOBC_ERR_CUDA;
    }
    // capture the whole launch sequence once (needs a capturable stream)
    if (b->stream) {
        cudaGraph_t graph = nullptr;
        err = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        hobc_status s = HOBC_OK;
        if (err == cudaSuccess) s = d.prec == HOBC_FP64 ? launch_all<double>(b) : launch_all<float>(b);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (err == cudaSuccess) err = e2;
        if (err == cudaSuccess && s == HOBC_OK) err = cudaGraphInstantiate(&b->graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (err != cudaSuccess || s != HOBC_OK) {
            if (err != cudaSuccess) set_last_error("hobc_batch_create: graph capture", err);
            hobc_batch_destroy(b);
            return err != cudaSuccess ? HOBC_ERR_CUDA : s;
        }
    }
    *out = b;
    return HOBC_OK;
}

extern "C" hobc_status hobc_batch_create(const hobc_batch_desc* desc, const hobc_batch_item* items,
                                         const double* mu_grid_host, void* cuda_stream, hobc_batch** out) {
    return hobc_batch_create_tuned(desc, items, mu_grid_host, nullptr, 0, cuda_stream, out);
}

extern "C" hobc_status hobc_batch_offsets(const hobc_batch* b, size_t* img_off, size_t* psf_off) {
    if (!b) return HOBC_ERR_ARG;
    if (img_off) std::copy(b->img_off.begin(), b->img_off.end(), img_off);
    if (psf_off) std::copy(b->psf_off.begin(), b->psf_off.end(), psf_off);
    return HOBC_OK;
}

extern "C" int hobc_batch_launch_count(const hobc_batch* b) { return b ? b->launches : 0; }

extern "C" hobc_status hobc_deblur_batched(hobc_batch* b, const void* g_dev, const void* psf_dev, void* f_dev,
                                           int* mu_index_dev, double* gcv_dev) {
    if (!b || !g_dev || !psf_dev || !f_dev) return HOBC_ERR_ARG;
    BatchIO io;
    io.g = g_dev;
    io.psf = psf_dev;
    io.f = f_dev;
    io.mu_idx = mu_index_dev ? mu_index_dev : b->mu_idx_ws;
    io.gcv = gcv_dev;
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    cudaError_t e = cudaMemcpyAsync(b->io_dev, &io, sizeof(io), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) { set_last_error("hobc_deblur_batched", e); return HOBC_ERR_CUDA; }
    if (b->graph) {
        e = cudaGraphLaunch(b->graph, b->stream);
        if (e != cudaSuccess) { set_last_error("hobc_deblur_batched: graph launch", e); return HOBC_ERR_CUDA; }
        return HOBC_OK;
    }
    return b->prec == HOBC_FP64 ? launch_all<double>(b) : launch_all<float>(b);
}
