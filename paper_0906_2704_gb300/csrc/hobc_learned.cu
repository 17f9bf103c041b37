// Learned choice of mu (an extension; the paper has no counterpart): a small
// MLP predicts log10(mu_GCV) from the radial spectra of ghat and d, the GCV
// functional is evaluated at the prediction and at the nearest +-4 grid
// values only, and a problem falls back to the full GCV scan when the
// prediction raises G by more than 5% over that bracket or the bracket
// minimum sits on its edge.  Everything runs in the kernels below: features,
// the network's forward and backward passes (tiled FP32-accumulating GEMMs
// with BF16 weights), AdamW, the bracket scan and the masked full scan.
// The same bracket scan serves the binned choice of mu (include/hobc_binned.h)
// and the continuous refinement of mu* (include/hobc_refine.h).
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/hobc_binned.h"
#include "../../include/hobc_learned.h"
#include "../../include/hobc_refine.h"
#include "hobc_internal.h"
#include "hobc_kernels.cuh"

namespace hobc {

constexpr int kBins = 64;            // radial bins per spectrum
constexpr int kFeat = 2 * kBins;     // network inputs
static_assert(kBins == 64, "k_features gives each lane of a warp two bins");
constexpr int kJ = 10;               // bracket slots of the binned choice and the refinement: mu_hat and up to 9 grid values
constexpr int kJL = 18;              // bracket slots of the learned choice: mu_hat and up to 17 grid values
constexpr int kBracketChunk = 4096;  // spectral entries per bracket-scan CTA
constexpr int kBracketU = 4;         // entries per thread whose loads are issued together

// ------------------------------------------------------------ features

// theta_t / pi of an axis as the exact fraction a / q, folded into [0, 1] (the
// Fourier family's angles run over [0, 2 pi)); border columns have a = 0.
__device__ __forceinline__ void angle_fraction(int fam, int n, int t, long long& a, long long& q) {
    if (fam == FAM_S) { q = n - 1; a = (t == n - 1) ? 0 : t; return; }
    const bool border = t == 0 || t == n - 1 || ((fam == FAM_S3 || fam == FAM_C4) && (t == 1 || t == n - 2));
    if (fam == FAM_S3) { q = n - 3; a = border ? 0 : t - 1; return; }
    if (fam == FAM_C4) { q = n - 4; a = border ? 0 : t - 2; return; }
    q = n - 2;
    if (border) { a = 0; return; }
    a = (fam == FAM_F) ? 2LL * (t - 1) : (long long)(t - 1);
    if (a > q) a = 2 * q - a;
}

// Radial bin floor(kBins * rho), rho^2 = (f0^2 + f1^2) / 2, decided exactly in
// integers: the largest b with b^2 q0^2 q1^2 <= (kBins^2 / 2)(a0^2 q1^2 + a1^2 q0^2).
__device__ __forceinline__ int radial_bin(long long a0, long long q0, long long a1, long long q1) {
    const long long Y = q0 * q0 * q1 * q1;
    const long long X = (long long)(kBins * kBins / 2) * (a0 * a0 * q1 * q1 + a1 * a1 * q0 * q0);
    int b = (int)sqrtf((float)X / (float)Y);
    while (b > 0 && (long long)b * b * Y > X) --b;
    while ((long long)(b + 1) * (b + 1) * Y <= X) ++b;
    return b < kBins - 1 ? b : kBins - 1;
}

// Per plan: the bin of every stored spectral entry (bits 0-5) and whether it
// stands for a conjugate pair of the Fourier half spectrum (bit 6, weight 2).
// grid-stride over the S entries of one item (all items share the geometry).
__global__ void k_bin_table(GcvGeom geo, int cplx, unsigned char* __restrict__ tab) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < geo.S;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / geo.n0), t0 = (int)(e - (long long)c * geo.n0);
        const int t1 = stored_to_t(geo.fam, geo.n1, geo.W1, c);
        long long a0, q0, a1, q1;
        angle_fraction(geo.fam, geo.n0, t0, a0, q0);
        angle_fraction(geo.fam, geo.n1, t1, a1, q1);
        const int b = radial_bin(a0, q0, a1, q1);
        const bool pair = cplx && !(c == 0 || c == geo.W1 - 1 || c == 1 || 2 * (c - 1) == geo.N1);
        tab[e] = (unsigned char)(b | (pair ? 64 : 0));
    }
}

// Per-CTA sums of weight, w|ghat|^2 and w|d|^2 in each radial bin, in a fixed
// order (the same input gives the same features bit for bit).  Each warp walks
// its share of the chunk 32 entries at a time: lanes holding consecutive
// entries of one bin form a run, a segmented scan sums each run into its last
// lane, and the run totals are added to the warp's own bins in lane order.
// The eight warps' bins are then combined in warp order.
// grid = items x ceil(S / kFeatChunk), block = 256; partials [CTA][3][kBins].
template <typename T, bool CPLX>
__global__ void __launch_bounds__(256)
k_features(const typename ElemT<T, CPLX>::t* __restrict__ spec, const typename ElemT<T, CPLX>::t* __restrict__ D,
           long long d_psf_stride, int psf_per, long long S, int chunk, const unsigned char* __restrict__ tab,
           double* __restrict__ partials) {
    __shared__ float ws[8][3][kBins];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    for (int k = lane; k < 3 * kBins; k += 32) ws[warp][k / kBins][k % kBins] = 0.f;
    __syncwarp();
    const int nch = (int)((S + chunk - 1) / chunk);
    const long long item = blockIdx.x / nch;
    const int ci = blockIdx.x - (int)(item * nch);
    const long long e0 = (long long)ci * chunk;
    const int cnt = (int)min((long long)chunk, S - e0);
    const typename ElemT<T, CPLX>::t* sp = spec + item * S + e0;
    const typename ElemT<T, CPLX>::t* dp = D + (psf_per ? item : 0) * d_psf_stride + e0;
    const int per_warp = (cnt + 7) / 8;
    const int w0 = warp * per_warp, w1 = min(cnt, w0 + per_warp);
    for (int base = w0; base < w1; base += 32) {
        const int i = base + lane;
        const bool valid = i < w1;
        int key = -1 - lane;                          // never equal to a neighbour's
        float vc = 0.f, vg = 0.f, vd = 0.f;
        if (valid) {
            const unsigned char tb = tab[e0 + i];
            key = tb & 63;
            vc = (tb & 64) ? 2.f : 1.f;
            vg = vc * (float)abs2_of(sp[i]);
            vd = vc * (float)abs2_of(dp[i]);
        }
        // runs of equal neighbouring keys, numbered in lane order
        const int prev = __shfl_up_sync(FULL, key, 1);
        const bool head = lane == 0 || prev != key;
        const unsigned heads = __ballot_sync(FULL, head);
        const int run = __popc(heads & (0xffffffffu >> (31 - lane)));   // heads in lanes 0..lane
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int r = __shfl_up_sync(FULL, run, d);
            const float a = __shfl_up_sync(FULL, vc, d);
            const float b = __shfl_up_sync(FULL, vg, d);
            const float c = __shfl_up_sync(FULL, vd, d);
            if (lane >= d && r == run) { vc += a; vg += b; vd += c; }
        }
        const int next = __shfl_down_sync(FULL, run, 1);
        const bool tail = valid && (lane == 31 || next != run);
        const unsigned tails = __ballot_sync(FULL, tail);
        if (tail) {
            const unsigned same = __match_any_sync(tails, key);     // tails of other runs of this bin
            const int rank = __popc(same & ((1u << lane) - 1u));
            const int rounds = __reduce_max_sync(tails, (unsigned)__popc(same));
            for (int r = 0; r < rounds; ++r) {
                if (rank == r) {
                    ws[warp][0][key] += vc;
                    ws[warp][1][key] += vg;
                    ws[warp][2][key] += vd;
                }
                __syncwarp(tails);
            }
        }
        __syncwarp();
    }
    __syncthreads();
    double* o = partials + (long long)blockIdx.x * 3 * kBins;
    for (int k = threadIdx.x; k < 3 * kBins; k += blockDim.x) {
        double acc = 0;
        for (int v = 0; v < 8; ++v) acc += ws[v][k / kBins][k % kBins];
        o[k] = acc;
    }
}

__global__ void k_features_finalize(const double* __restrict__ partials, int nchunks, float* __restrict__ X) {
    const int item = blockIdx.x;
    const double* p = partials + (long long)item * nchunks * 3 * kBins;
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) {
        double c = 0, g = 0, d = 0;
        for (int k = 0; k < nchunks; ++k) {
            c += p[(long long)k * 3 * kBins + b];
            g += p[(long long)k * 3 * kBins + kBins + b];
            d += p[(long long)k * 3 * kBins + 2 * kBins + b];
        }
        X[(long long)item * kFeat + b] = (float)log10((c > 0 ? g / c : 0.0) + 1e-30);
        X[(long long)item * kFeat + kBins + b] = (float)log10((c > 0 ? d / c : 0.0) + 1e-30);
    }
}

// ------------------------------------------------------------------ MLP

__device__ __forceinline__ float ldf(float x) { return x; }
__device__ __forceinline__ float ldf(__nv_bfloat16 x) { return __bfloat162float(x); }

__device__ __forceinline__ __nv_bfloat16 to_bf16(float x) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ __nv_bfloat16 to_bf16(__nv_bfloat16 x) { return x; }

// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]); A(m,k) = TRA ? A[k lda + m] : A[m lda + k],
// B(k,n) = TRB ? B[n ldb + k] : B[k ldb + n].  On the tensor cores: both
// operands rounded to bfloat16 (nearest, ties to even) as they are staged in
// shared memory, mma.sync m16n8k16 with FP32 accumulation.  64x64 tiles, K
// steps of 16; 4 warps, each a 32x32 quarter (2 x 4 MMA tiles of 16x8).
template <typename TA, typename TB, bool TRA, bool TRB>
__global__ void __launch_bounds__(128)
k_gemm(int M, int N, int K, const TA* __restrict__ A, int lda, const TB* __restrict__ B, int ldb,
       float* __restrict__ C, int ldc, const float* __restrict__ bias) {
    constexpr int LD = 16 + 8;                   // bf16 per tile row: k pairs stay 4-byte aligned
    __shared__ __align__(16) __nv_bfloat16 As[64][LD];   // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[64][LD];   // [n][k]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane >> 2, tig = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[2][4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int l = threadIdx.x; l < 1024; l += 128) {
            int mm, kk;
            if (TRA) { kk = l / 64; mm = l % 64; } else { mm = l / 16; kk = l % 16; }
            const int m = m0 + mm, k = k0 + kk;
            __nv_bfloat16 v = __float2bfloat16_rn(0.f);
            if (m < M && k < K) v = to_bf16(TRA ? A[(long long)k * lda + m] : A[(long long)m * lda + k]);
            As[mm][kk] = v;
        }
        for (int l = threadIdx.x; l < 1024; l += 128) {
            int kk, nn;
            if (TRB) { nn = l / 16; kk = l % 16; } else { kk = l / 64; nn = l % 64; }
            const int n = n0 + nn, k = k0 + kk;
            __nv_bfloat16 v = __float2bfloat16_rn(0.f);
            if (n < N && k < K) v = to_bf16(TRB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n]);
            Bs[nn][kk] = v;
        }
        __syncthreads();
        uint32_t af[2][4], bfr[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm + 16 * i + grp;
            af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][2 * tig]);
            af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][2 * tig]);
            af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][2 * tig + 8]);
            af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][2 * tig + 8]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = wn + 8 * j + grp;
            bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][2 * tig]);
            bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][2 * tig + 8]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                    : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                    : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]), "r"(bfr[j][1]));
        __syncthreads();
    }
    // accumulator (i, j): rows grp, grp + 8 of the 16x8 tile, columns 2 tig, 2 tig + 1
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int m = m0 + wm + 16 * i + grp + (h >> 1) * 8;
                const int n = n0 + wn + 8 * j + 2 * tig + (h & 1);
                if (m < M && n < N) C[(long long)m * ldc + n] = acc[i][j][h] + (bias ? bias[n] : 0.f);
            }
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

__global__ void k_standardize(const float* __restrict__ x, const float* __restrict__ mean,
                              const float* __restrict__ scale, float* __restrict__ xs, long long count, int nin) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i % nin);
        xs[i] = (x[i] - mean[f]) / scale[f];
    }
}

__global__ void k_gelu(const float* __restrict__ z, float* __restrict__ h, long long count) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
        h[i] = gelu_f(z[i]);
}

// y[b] = h2[b] . w3 + b3, one warp per sample
__global__ void k_output(const float* __restrict__ h2, const __nv_bfloat16* __restrict__ w3, const float* __restrict__ b3,
                         float* __restrict__ y, int B, int nh) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
    if (warp >= B) return;
    float acc = 0.f;
    for (int o = lane; o < nh; o += 32) acc = fmaf(h2[(long long)warp * nh + o], __bfloat162float(w3[o]), acc);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) y[warp] = acc + b3[0];
}

// dy = 2 (y - t) / B and the mean squared error (one block)
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, int B, float* __restrict__ dy,
                       float* __restrict__ loss) {
    __shared__ double s[256];
    double acc = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float r = y[b] - t[b];
        dy[b] = 2.f * r / B;
        acc += (double)r * r;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) loss[0] = (float)(s[0] / B);
}

// dz2[b][o] = dy[b] w3[o] GELU'(z2[b][o])
__global__ void k_dz_out(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ w3, const float* __restrict__ z2,
                         float* __restrict__ dz2, int B, int nh) {
    const long long count = (long long)B * nh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / nh), o = (int)(i % nh);
        dz2[i] = dy[b] * __bfloat162float(w3[o]) * gelu_grad_f(z2[i]);
    }
}

__global__ void k_gelu_bwd(const float* __restrict__ dh, const float* __restrict__ z, float* __restrict__ dz, long long count) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
        dz[i] = dh[i] * gelu_grad_f(z[i]);
}

// out[o] = sum_b A[b][o] (* w[b] if given)
__global__ void k_colsum(const float* __restrict__ A, const float* __restrict__ w, int B, int nh, float* __restrict__ out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nh) return;
    float acc = 0.f;
    for (int b = 0; b < B; ++b) acc = fmaf(A[(long long)b * nh + o], w ? w[b] : 1.f, acc);
    out[o] = acc;
}

__global__ void k_sum(const float* __restrict__ v, int B, float* __restrict__ out) {
    __shared__ float s[256];
    float acc = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) acc += v[b];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0];
}

__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                        int P, float lr, float b1, float b2, float eps, float wd, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
    }
}

// Per input feature j (one CTA each): mean and standard deviation of column j
// of x [rows][nin] in FP64, two passes, fixed-order tree sums; scale = std +
// 1e-3.  grid = nin, block = 256.
__global__ void k_fit_scaling(const float* __restrict__ x, int rows, int nin, float* __restrict__ mean,
                              float* __restrict__ scale) {
    __shared__ double red[256];
    const int j = blockIdx.x;
    double acc = 0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) acc += (double)x[(long long)r * nin + j];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double mu = red[0] / rows;
    __syncthreads();
    acc = 0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const double dlt = (double)x[(long long)r * nin + j] - mu;
        acc += dlt * dlt;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mean[j] = (float)mu;
        scale[j] = (float)(sqrt(red[0] / rows) + 1e-3);
    }
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ q, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) q[i] = __float2bfloat16_rn(p[i]);
}

// ----------------------------------------------------- learned deblurring

// mu lists of the bracket check, kJ wide: [mu_hat, grid[k0 .. k0 + J - 2]], k0
// around the grid index nearest to mu_hat (in log10), clamped to the grid;
// entries past J repeat the last one.
template <typename T, int JS>
__global__ void k_bracket_setup(const float* __restrict__ y, const double* __restrict__ grid,
                                const double* __restrict__ lg, int K, int J, T* __restrict__ lists,
                                double* __restrict__ mu_hat, int* __restrict__ k0_out, int B) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= B) return;
    const double yv = (double)y[item];
    const double l = (yv == yv) ? fmin(fmax(yv, lg[0]), lg[K - 1]) : lg[0];   // NaN -> grid start
    const double mh = pow(10.0, l);
    int lo = 0, hi = K - 1;                      // first k with lg[k] >= l (lg increasing)
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (lg[mid] >= l) hi = mid; else lo = mid + 1;
    }
    int kn = lo;
    if (kn > 0 && fabs(lg[kn - 1] - l) <= fabs(lg[kn] - l)) kn = kn - 1;   // nearest, lower index on ties
    const int span = J - 1;
    int k0 = kn - span / 2;
    k0 = max(0, min(k0, K - span));
    mu_hat[item] = mh;
    k0_out[item] = k0;
    T* o = lists + (long long)item * JS;
    o[0] = (T)mh;
    for (int j = 1; j < JS; ++j) o[j] = (T)grid[k0 + min(j, J - 1) - 1];
}

// G at the bracket values: accept mu_hat unless it raises G by more than 5% over
// the bracket minimum or that minimum is on an edge that is not the grid's end.
__global__ void k_bracket_decide(const double* __restrict__ Gb, int J, int JS, const int* __restrict__ k0, int K,
                                 const double* __restrict__ mu_hat, double* __restrict__ mu_val,
                                 int* __restrict__ fell_back, int B) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= B) return;
    const double* g = Gb + (long long)item * JS;
    double mn = INFINITY;
    int am = 1;
    for (int j = 1; j < J; ++j)
        if (g[j] < mn) { mn = g[j]; am = j; }
    const int kmin = k0[item] + am - 1;
    const bool edge = (am == 1 && kmin > 0) || (am == J - 1 && kmin < K - 1);
    const bool worse = !(g[0] <= 1.05 * mn);           // also catches NaN
    const int fb = (edge || worse) ? 1 : 0;
    fell_back[item] = fb;
    mu_val[item] = mu_hat[item];
}

// G's sums at the JS bracket values of every problem: each thread takes its
// elements' terms once and accumulates all JS values (reciprocals shared by
// pairs, as in the grid scan); sums per thread and per warp in T, across
// warps in double.
// grid = items x ceil(S / kBracketChunk), block = 256; partials [CTA][2 JS].
template <typename T, bool CPLX, int JS = kJ>
__global__ void __launch_bounds__(256)
k_gcv_bracket(const typename ElemT<T, CPLX>::t* __restrict__ spec, const typename ElemT<T, CPLX>::t* __restrict__ D,
              long long d_psf_stride, int psf_per, const T* __restrict__ lists, GcvGeom geo,
              double* __restrict__ partials) {
    __shared__ double red[8][2 * JS];
    const int nch = (int)((geo.S + kBracketChunk - 1) / kBracketChunk);
    const long long item = blockIdx.x / nch;
    const int chunk = blockIdx.x - (int)(item * nch);
    const long long e0 = (long long)chunk * kBracketChunk;
    const int cnt = (int)min((long long)kBracketChunk, geo.S - e0);
    const typename ElemT<T, CPLX>::t* sp = spec + item * geo.S + e0;
    const typename ElemT<T, CPLX>::t* dp = D + (psf_per ? item : 0) * d_psf_stride + e0;
    T mu[JS], nd[JS], dd[JS];
#pragma unroll
    for (int j = 0; j < JS; ++j) { mu[j] = lists[item * JS + j]; nd[j] = 0; dd[j] = 0; }
    // kBracketU entries per thread and step, all loads issued before the math:
    // with ten evaluations per entry the pass is bound by load latency
    typedef typename ElemT<T, CPLX>::t E;
    for (int i0 = threadIdx.x; i0 < cnt; i0 += kBracketU * blockDim.x) {
        E sv[kBracketU], dv[kBracketU];
#pragma unroll
        for (int u = 0; u < kBracketU; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < cnt) { sv[u] = sp[i]; dv[u] = dp[i]; }
        }
#pragma unroll
        for (int u = 0; u < kBracketU; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i >= cnt) break;
            const typename Pack4<T>::t v = gcv_term<T, CPLX>(sv[u], dv[u], geo, e0 + i);
#pragma unroll
            for (int j = 0; j < JS; j += 2) {
                const T t1 = v.x + mu[j], t2 = v.x + mu[j + 1];
                const T r = pair_rcp(t1 * t2);
                const T s1 = t2 * r, s2 = t1 * r;
                dd[j] += v.z * s1;
                dd[j + 1] += v.z * s2;
                nd[j] += v.y * s1 * s1;
                nd[j + 1] += v.y * s2 * s2;
            }
        }
    }
    // warp sums in the working precision (a thread holds at most
    // kBracketChunk / 256 entries, so at most 16 + 5 roundings in FP32), one
    // conversion per warp: FP64 runs at a small fraction of the FP32 rate
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
    for (int j = 0; j < JS; ++j) {
        T a = nd[j], b = dd[j];
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, off);
            b += __shfl_down_sync(0xffffffffu, b, off);
        }
        if (lane == 0) { red[warp][j] = (double)a; red[warp][JS + j] = (double)b; }
    }
    __syncthreads();
    if (threadIdx.x < 2 * JS) {
        double acc = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) acc += red[w][threadIdx.x];
        partials[(long long)blockIdx.x * 2 * JS + threadIdx.x] = acc;
    }
}

// G at the JS bracket values of every problem from the per-CTA sums: 256 / (2 JS)
// groups of 2 JS threads split the chunks, then combine in group order.
// grid = items, block = 256; G [item][JS].
template <int JS = kJ>
__global__ void k_bracket_finalize(const double* __restrict__ partials, int nchunks, double* __restrict__ G) {
    constexpr int V = 2 * JS, NG = 256 / V;
    __shared__ double acc[NG][V];
    const int item = blockIdx.x;
    const int g = threadIdx.x / V, v = threadIdx.x % V;
    if (g < NG) {
        double a = 0;
        for (int c = g; c < nchunks; c += NG) a += partials[((long long)item * nchunks + c) * V + v];
        acc[g][v] = a;
    }
    __syncthreads();
    if (threadIdx.x < JS) {
        double num = 0, den = 0;
        for (int q = 0; q < NG; ++q) { num += acc[q][threadIdx.x]; den += acc[q][JS + threadIdx.x]; }
        G[(long long)item * JS + threadIdx.x] = num / (den * den);
    }
}

// ------------------------------------------- continuous refinement of mu*
// Eq. (eq:mugcv) minimises G over mu > 0; the grid argmin k only brackets the
// minimiser.  Per problem the search keeps lo, mid, hi in log10 mu and the
// incumbent mu (the value G was evaluated at).  Every round evaluates G at
// nine points, four equal log10 steps from lo to mid and four from mid to hi
// (point 4 is the incumbent, point 9 of the kJ slots repeats point 8), moves
// mid to the first minimiser j (NaN never wins; all NaN keeps the incumbent)
// and lo, hi to its neighbours.  Rounds shrink the bracket about four times.
constexpr int kRefinePoints = 9;
constexpr int kRefineRounds = 5;
static_assert(kRefinePoints <= kJ, "a round's points fit the bracket scan's slots");

__device__ __forceinline__ double refine_point(double lo, double mid, double hi, int j) {
    constexpr int half = kRefinePoints / 2;
    return j <= half ? lo + (mid - lo) * j / half : mid + (hi - mid) * (j - half) / half;
}

template <typename T>
__device__ __forceinline__ void refine_lists(double lo, double mid, double hi, double mid_mu, T* o) {
    for (int j = 0; j < kRefinePoints; ++j)
        o[j] = j == kRefinePoints / 2 ? (T)mid_mu : (T)pow(10.0, refine_point(lo, mid, hi, j));
    for (int j = kRefinePoints; j < kJ; ++j) o[j] = o[kRefinePoints - 1];
}

// Round 0 around the grid argmin: st[item] = (lo, mid, hi, incumbent mu).
template <typename T>
__global__ void k_refine_init(const int* __restrict__ mu_idx, const double* __restrict__ grid,
                              const double* __restrict__ lg, int K, double* __restrict__ st, T* __restrict__ lists,
                              int B) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= B) return;
    const int k = min(max(mu_idx[item], 0), K - 1);
    const double lo = lg[max(k - 1, 0)], mid = lg[k], hi = lg[min(k + 1, K - 1)];
    const double mid_mu = (double)(T)grid[k];
    double* q = st + 4LL * item;
    q[0] = lo; q[1] = mid; q[2] = hi; q[3] = mid_mu;
    refine_lists<T>(lo, mid, hi, mid_mu, lists + (long long)item * kJ);
}

// After a round's G: the next round's bracket and points, or (last round) mu*
// and G(mu*).
template <typename T>
__global__ void k_refine_step(const double* __restrict__ Gb, double* __restrict__ st, T* __restrict__ lists,
                              int last, double* __restrict__ mu_out, double* __restrict__ G_out, int B) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= B) return;
    const double* g = Gb + (long long)item * kJ;
    int jm = kRefinePoints / 2;
    double best = INFINITY;
    bool any = false;
    for (int j = 0; j < kRefinePoints; ++j) {
        if (isnan(g[j])) continue;
        if (!any || g[j] < best) { best = g[j]; jm = j; any = true; }
    }
    double* q = st + 4LL * item;
    const double lo = q[0], mid = q[1], hi = q[2];
    T* o = lists + (long long)item * kJ;
    const double mu_j = (double)o[jm];
    if (last) {
        mu_out[item] = mu_j;
        if (G_out) G_out[item] = g[jm];
        return;
    }
    const double nlo = refine_point(lo, mid, hi, max(jm - 1, 0));
    const double nmid = refine_point(lo, mid, hi, jm);
    const double nhi = refine_point(lo, mid, hi, min(jm + 1, kRefinePoints - 1));
    q[0] = nlo; q[1] = nmid; q[2] = nhi; q[3] = mu_j;
    refine_lists<T>(nlo, nmid, nhi, mu_j, o);
}

template <typename T, bool CPLX>
__global__ void __launch_bounds__(256)
k_gcv_masked(const typename ElemT<T, CPLX>::t* __restrict__ spec, const typename ElemT<T, CPLX>::t* __restrict__ D,
             long long d_psf_stride, int psf_per, const T* __restrict__ muT, GcvGeom geo, const int* __restrict__ mask,
             double* __restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nch = (int)((geo.S + geo.chunk - 1) / geo.chunk);
    const long long item = blockIdx.x / nch;
    if (!mask[item]) return;
    const int chunk = blockIdx.x - (int)(item * nch);
    gcv_partials_body<T, CPLX>(spec + item * geo.S, D + (psf_per ? item : 0) * d_psf_stride, muT, geo,
                               (long long)chunk * geo.chunk, partials + (long long)blockIdx.x * 2LL * geo.K, smem_raw);
}

// argmin over the full grid for the problems that fell back; mu_val = grid[argmin]
__global__ void k_masked_finalize(const double* __restrict__ partials, int nchunks, int K, const int* __restrict__ mask,
                                  const double* __restrict__ grid, double* __restrict__ mu_val,
                                  int* __restrict__ mu_idx) {
    __shared__ double sv[256];
    __shared__ int si[256];
    const int item = blockIdx.x;
    if (!mask[item]) return;
    const double* p = partials + (long long)item * nchunks * 2 * K;
    double best = INFINITY;
    int bi = 0x7fffffff;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        double num, den;
        sum_chunks(p, nchunks, K, j, num, den);
        const double Gv = num / (den * den);
        const double key = isnan(Gv) ? INFINITY : Gv;
        if (key < best || (key == best && j < bi)) { best = key; bi = j; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            if (sv[threadIdx.x + s] < sv[threadIdx.x] ||
                (sv[threadIdx.x + s] == sv[threadIdx.x] && si[threadIdx.x + s] < si[threadIdx.x])) {
                sv[threadIdx.x] = sv[threadIdx.x + s];
                si[threadIdx.x] = si[threadIdx.x + s];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int k = si[0] == 0x7fffffff ? 0 : si[0];
        if (mu_val) mu_val[item] = grid[k];
        if (mu_idx) mu_idx[item] = k;
    }
}

// ------------------------------------------------------------- binned choice

constexpr int kABins = 128;          // bins of log10 a over [1e-12, 1e4)
constexpr int kAChunk = 16384;       // spectral entries per histogram CTA (2048 per warp)
constexpr double kALo = -12.0, kAHi = 4.0;

// Per-CTA histogram of the GCV terms over a = |d|^2/|s|^2: per bin the weight
// W, the energy E = w |ghat|^2 and A = w a.  An entry's bin is the number of
// interior edges <= a (end bins take everything outside); entries with s = 0
// are left out.  Same deterministic warp reduction as k_features.
// grid = items x ceil(S / geo.chunk), block = 256; partials [CTA][3][kABins].
template <typename T, bool CPLX>
__global__ void __launch_bounds__(256)
k_ahist(const typename ElemT<T, CPLX>::t* __restrict__ spec, const typename ElemT<T, CPLX>::t* __restrict__ D,
        long long d_psf_stride, int psf_per, GcvGeom geo, const T* __restrict__ edges,
        double* __restrict__ partials) {
    __shared__ float ws[8][3][kABins];
    __shared__ T ed[kABins + 1];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    for (int k = threadIdx.x; k <= kABins; k += blockDim.x) ed[k] = edges[k];
    for (int k = lane; k < 3 * kABins; k += 32) ws[warp][k / kABins][k % kABins] = 0.f;
    __syncthreads();
    const int nch = (int)((geo.S + geo.chunk - 1) / geo.chunk);
    const long long item = blockIdx.x / nch;
    const int ci = blockIdx.x - (int)(item * nch);
    const long long e0 = (long long)ci * geo.chunk;
    const int cnt = (int)min((long long)geo.chunk, geo.S - e0);
    const typename ElemT<T, CPLX>::t* sp = spec + item * geo.S + e0;
    const typename ElemT<T, CPLX>::t* dp = D + (psf_per ? item : 0) * d_psf_stride + e0;
    const int per_warp = (cnt + 7) / 8;
    const int w0 = warp * per_warp, w1 = min(cnt, w0 + per_warp);
    for (int base = w0; base < w1; base += 32) {
        const int i = base + lane;
        bool valid = i < w1;
        int key = -1 - lane;
        float vc = 0.f, vg = 0.f, va = 0.f;
        if (valid) {
            const typename Pack4<T>::t v = gcv_term<T, CPLX>(sp[i], dp[i], geo, e0 + i);
            valid = v.z > (T)0;
            if (valid) {
                // estimate the bin from log10 a, then settle it exactly against the
                // edges: the bin is the number of interior edges <= a
                float la = __log2f((float)v.x) * 0.30102999566f;
                la = fminf(fmaxf(la, (float)kALo - 1.f), (float)kAHi + 1.f);
                int b = (int)floorf((la - (float)kALo) * (float)(kABins / (kAHi - kALo)));
                b = min(max(b, 0), kABins - 1);
                while (b > 0 && v.x < ed[b]) --b;
                while (b < kABins - 1 && v.x >= ed[b + 1]) ++b;
                key = b;
                vc = (float)v.z;
                vg = (float)v.y;
                va = (float)(v.z * v.x);
            }
        }
        const int prev = __shfl_up_sync(FULL, key, 1);
        const bool head = lane == 0 || prev != key;
        const unsigned heads = __ballot_sync(FULL, head);
        const int run = __popc(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int r = __shfl_up_sync(FULL, run, d);
            const float a = __shfl_up_sync(FULL, vc, d);
            const float b = __shfl_up_sync(FULL, vg, d);
            const float c = __shfl_up_sync(FULL, va, d);
            if (lane >= d && r == run) { vc += a; vg += b; va += c; }
        }
        const int next = __shfl_down_sync(FULL, run, 1);
        const bool tail = valid && (lane == 31 || next != run);
        const unsigned tails = __ballot_sync(FULL, tail);
        if (tail) {
            const unsigned same = __match_any_sync(tails, key);
            const int rank = __popc(same & ((1u << lane) - 1u));
            const int rounds = __reduce_max_sync(tails, (unsigned)__popc(same));
            for (int r = 0; r < rounds; ++r) {
                if (rank == r) {
                    ws[warp][0][key] += vc;
                    ws[warp][1][key] += vg;
                    ws[warp][2][key] += va;
                }
                __syncwarp(tails);
            }
        }
        __syncwarp();
    }
    __syncthreads();
    double* o = partials + (long long)blockIdx.x * 3 * kABins;
    for (int k = threadIdx.x; k < 3 * kABins; k += blockDim.x) {
        double acc = 0;
        for (int v = 0; v < 8; ++v) acc += ws[v][k / kABins][k % kABins];
        o[k] = acc;
    }
}

// Per problem: the bin sums over all chunks, G_bin(mu_j) for every grid value
// (normalised energies and weights, FP32 terms, 1/(abar + mu) with abar + mu
// kept >= 1e-18), its first minimiser k_hat (NaN never wins), and the bracket
// of min(9, K) grid values around k_hat as the list of the exact scan.
// grid = items, block = 256.
template <typename T>
__global__ void k_binned_khat(const double* __restrict__ partials, int nchunks, const double* __restrict__ grid, int K,
                              int* __restrict__ k_hat, int* __restrict__ k0_out, T* __restrict__ lists) {
    __shared__ float sa[kABins], se[kABins], sw[kABins];
    __shared__ double rmax[kABins], rsum[kABins];
    __shared__ float sv[256];
    __shared__ int si[256];
    const int item = blockIdx.x;
    __shared__ double sum3[3 * kABins];
    const double* p = partials + (long long)item * nchunks * 3 * kABins;
    for (int k = threadIdx.x; k < 3 * kABins; k += blockDim.x) {   // chunk sums, four loads in flight
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int c = 0;
        for (; c + 4 <= nchunks; c += 4) {
            a0 += p[(long long)c * 3 * kABins + k];
            a1 += p[(long long)(c + 1) * 3 * kABins + k];
            a2 += p[(long long)(c + 2) * 3 * kABins + k];
            a3 += p[(long long)(c + 3) * 3 * kABins + k];
        }
        for (; c < nchunks; ++c) a0 += p[(long long)c * 3 * kABins + k];
        sum3[k] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    const double W = threadIdx.x < kABins ? sum3[threadIdx.x] : 0.0;
    const double E = threadIdx.x < kABins ? sum3[kABins + threadIdx.x] : 0.0;
    const double A = threadIdx.x < kABins ? sum3[2 * kABins + threadIdx.x] : 0.0;
    if (threadIdx.x < kABins) {
        rmax[threadIdx.x] = E;
        rsum[threadIdx.x] = W;
    }
    __syncthreads();
    for (int st = kABins / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            rmax[threadIdx.x] = fmax(rmax[threadIdx.x], rmax[threadIdx.x + st]);
            rsum[threadIdx.x] += rsum[threadIdx.x + st];
        }
        __syncthreads();
    }
    const double emax = rmax[0] > 0 ? rmax[0] : 1.0, wtot = rsum[0] > 0 ? rsum[0] : 1.0;
    if (threadIdx.x < kABins) {
        const int b = threadIdx.x;
        sa[b] = W > 0 ? (float)(A / W) : 1.f;
        se[b] = (float)(E / emax);
        sw[b] = (float)(W / wtot);
    }
    __syncthreads();
    float best = INFINITY;
    int bi = 0x7fffffff;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        const float mu = (float)grid[j];
        float num = 0.f, den = 0.f;
        for (int b = 0; b < kABins; ++b) {
            const float r = __frcp_rn(fmaxf(sa[b] + mu, 1e-18f));
            den = fmaf(sw[b], r, den);
            num = fmaf(se[b] * r, r, num);
        }
        const float G = (float)((double)num / ((double)den * (double)den));
        const float key = isnan(G) ? INFINITY : G;
        if (key < best || (key == best && j < bi)) { best = key; bi = j; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            if (sv[threadIdx.x + st] < sv[threadIdx.x] ||
                (sv[threadIdx.x + st] == sv[threadIdx.x] && si[threadIdx.x + st] < si[threadIdx.x])) {
                sv[threadIdx.x] = sv[threadIdx.x + st];
                si[threadIdx.x] = si[threadIdx.x + st];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int kh = si[0] == 0x7fffffff ? 0 : si[0];
        const int span = min(kJ - 1, K);
        const int k0 = max(0, min(kh - span / 2, K - span));
        k_hat[item] = kh;
        k0_out[item] = k0;
        T* o = lists + (long long)item * kJ;
        for (int j = 0; j < kJ; ++j) o[j] = (T)grid[k0 + min(j, span - 1)];
    }
}

// Histogram features of each problem (the learned choice's second feature
// kind): the chunk sums of k_ahist in chunk order, adjacent bins merged in
// pairs (kABins / 2 = kBins bins of 0.25 decade in log10 a), x[b] =
// log10(E_b / E + 1e-12) and x[kBins + b] = log10(W_b / W + 1e-12).
// grid = items, block = kABins.
__global__ void k_hist_features(const double* __restrict__ partials, int nchunks, float* __restrict__ X) {
    __shared__ double sw[kABins], se[kABins];
    __shared__ double tot[2];
    const int item = blockIdx.x, k = threadIdx.x;
    const double* p = partials + (long long)item * nchunks * 3 * kABins;
    double w = 0, e = 0;
    for (int c = 0; c < nchunks; ++c) {
        w += p[(long long)c * 3 * kABins + k];
        e += p[(long long)c * 3 * kABins + kABins + k];
    }
    sw[k] = w;
    se[k] = e;
    __syncthreads();
    if (k == 0) {
        double tw = 0, te = 0;
        for (int b = 0; b < kABins; ++b) { tw += sw[b]; te += se[b]; }
        tot[0] = tw;
        tot[1] = te;
    }
    __syncthreads();
    if (k < kBins) {
        const double eb = se[2 * k] + se[2 * k + 1], wb = sw[2 * k] + sw[2 * k + 1];
        X[(long long)item * 2 * kBins + k] = (float)log10(eb / tot[1] + 1e-12);
        X[(long long)item * 2 * kBins + kBins + k] = (float)log10(wb / tot[0] + 1e-12);
    }
}
static_assert(kABins == 2 * kBins, "feature bins merge pairs of histogram bins");

// The exact G on the bracket: its first minimiser is mu* unless it lies on a
// bracket edge that is not an end of the grid (then the problem falls back).
__global__ void k_binned_decide(const double* __restrict__ Gb, int K, const int* __restrict__ k0,
                                int* __restrict__ mu_idx, int* __restrict__ fell_back, int B) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= B) return;
    const int span = min(kJ - 1, K);
    const double* g = Gb + (long long)item * kJ;
    double mn = INFINITY;
    int am = 0;
    for (int j = 0; j < span; ++j)
        if (g[j] < mn) { mn = g[j]; am = j; }
    const int kmin = k0[item] + am;
    const bool edge = (am == 0 && kmin > 0) || (am == span - 1 && kmin < K - 1);
    fell_back[item] = edge ? 1 : 0;
    mu_idx[item] = kmin;
}

void free_learned_ws(hobc_plan_s* p) {
    void* ps[] = {p->feat_partials, p->feat, p->mlp_y, p->bracket_mu, p->mu_hat, p->bracket_k0,
                  p->bracket_partials, p->bracket_G, p->bracket_idx, p->mu_val, p->fell_back, p->log_grid,
                  p->bin_tab, p->ahist_partials, p->a_edges, p->k_hat, p->refine_state};
    for (void* q : ps) cudaFree(q);
    p->refine_state = nullptr;
    p->feat_partials = nullptr; p->feat = nullptr; p->mlp_y = nullptr; p->bracket_mu = nullptr;
    p->mu_hat = nullptr; p->bracket_k0 = nullptr; p->bracket_partials = nullptr; p->bracket_G = nullptr;
    p->bracket_idx = nullptr; p->mu_val = nullptr; p->fell_back = nullptr; p->log_grid = nullptr;
    p->bin_tab = nullptr; p->ahist_partials = nullptr; p->a_edges = nullptr; p->k_hat = nullptr;
}

}  // namespace hobc

using namespace hobc;

// =================================================================== MLP

struct hobc_mlp_s {
    int nin, nh, P, cap, step;
    int feature_kind;        // HOBC_FEATURES_RADIAL or HOBC_FEATURES_HIST: the inputs hobc_deblur_learned forms
    cudaStream_t stream;
    float *params, *grads, *m, *v, *mean, *scale;
    __nv_bfloat16 *w1h, *w2h, *w3h;
    float *xs, *z1, *h1, *z2, *h2, *y, *dy, *dz2, *dh1, *dz1, *loss;
    int launches;
};

namespace {

int oW1(const hobc_mlp_s* q) { return 0; }
int ob1(const hobc_mlp_s* q) { return q->nh * q->nin; }
int oW2(const hobc_mlp_s* q) { return ob1(q) + q->nh; }
int ob2(const hobc_mlp_s* q) { return oW2(q) + q->nh * q->nh; }
int ow3(const hobc_mlp_s* q) { return ob2(q) + q->nh; }
int ob3(const hobc_mlp_s* q) { return ow3(q) + q->nh; }

cudaError_t ensure_capacity(hobc_mlp_s* q, int B) {
    if (B <= q->cap) return cudaSuccess;
    float** bufs[] = {&q->xs, &q->z1, &q->h1, &q->z2, &q->h2, &q->dz2, &q->dh1, &q->dz1};
    for (float** b : bufs) { cudaFree(*b); *b = nullptr; }
    cudaFree(q->y); cudaFree(q->dy);
    cudaError_t e = cudaSuccess;
    const size_t wide = (size_t)B * std::max(q->nh, q->nin) * sizeof(float);
    for (float** b : bufs) if (e == cudaSuccess) e = cudaMalloc((void**)b, wide);
    if (e == cudaSuccess) e = cudaMalloc((void**)&q->y, (size_t)B * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&q->dy, (size_t)B * sizeof(float));
    if (e == cudaSuccess) q->cap = B;
    return e;
}

void refresh_bf16(hobc_mlp_s* q) {
    k_to_bf16<<<64, 256, 0, q->stream>>>(q->params + oW1(q), q->w1h, q->nh * q->nin);
    k_to_bf16<<<64, 256, 0, q->stream>>>(q->params + oW2(q), q->w2h, q->nh * q->nh);
    k_to_bf16<<<4, 256, 0, q->stream>>>(q->params + ow3(q), q->w3h, q->nh);
    q->launches += 3;
}

dim3 gemm_grid(int M, int N) { return dim3((N + 63) / 64, (M + 63) / 64); }

void forward(hobc_mlp_s* q, const float* x, int B, float* y_out) {
    cudaStream_t st = q->stream;
    const long long cx = (long long)B * q->nin, ch = (long long)B * q->nh;
    k_standardize<<<256, 256, 0, st>>>(x, q->mean, q->scale, q->xs, cx, q->nin);
    k_gemm<float, __nv_bfloat16, false, true><<<gemm_grid(B, q->nh), 128, 0, st>>>(
        B, q->nh, q->nin, q->xs, q->nin, q->w1h, q->nin, q->z1, q->nh, q->params + ob1(q));
    k_gelu<<<256, 256, 0, st>>>(q->z1, q->h1, ch);
    k_gemm<float, __nv_bfloat16, false, true><<<gemm_grid(B, q->nh), 128, 0, st>>>(
        B, q->nh, q->nh, q->h1, q->nh, q->w2h, q->nh, q->z2, q->nh, q->params + ob2(q));
    k_gelu<<<256, 256, 0, st>>>(q->z2, q->h2, ch);
    k_output<<<(B * 32 + 255) / 256, 256, 0, st>>>(q->h2, q->w3h, q->params + ob3(q), y_out, B, q->nh);
    q->launches += 6;
}

void backward(hobc_mlp_s* q, const float* t, int B, float* loss) {
    cudaStream_t st = q->stream;
    const long long ch = (long long)B * q->nh;
    float* g = q->grads;
    k_loss<<<1, 256, 0, st>>>(q->y, t, B, q->dy, loss);
    k_colsum<<<(q->nh + 255) / 256, 256, 0, st>>>(q->h2, q->dy, B, q->nh, g + ow3(q));
    k_sum<<<1, 256, 0, st>>>(q->dy, B, g + ob3(q));
    k_dz_out<<<256, 256, 0, st>>>(q->dy, q->w3h, q->z2, q->dz2, B, q->nh);
    k_gemm<float, float, true, false><<<gemm_grid(q->nh, q->nh), 128, 0, st>>>(
        q->nh, q->nh, B, q->dz2, q->nh, q->h1, q->nh, g + oW2(q), q->nh, nullptr);
    k_colsum<<<(q->nh + 255) / 256, 256, 0, st>>>(q->dz2, nullptr, B, q->nh, g + ob2(q));
    k_gemm<float, __nv_bfloat16, false, false><<<gemm_grid(B, q->nh), 128, 0, st>>>(
        B, q->nh, q->nh, q->dz2, q->nh, q->w2h, q->nh, q->dh1, q->nh, nullptr);
    k_gelu_bwd<<<256, 256, 0, st>>>(q->dh1, q->z1, q->dz1, ch);
    k_gemm<float, float, true, false><<<gemm_grid(q->nh, q->nin), 128, 0, st>>>(
        q->nh, q->nin, B, q->dz1, q->nh, q->xs, q->nin, g + oW1(q), q->nin, nullptr);
    k_colsum<<<(q->nh + 255) / 256, 256, 0, st>>>(q->dz1, nullptr, B, q->nh, g + ob1(q));
    q->launches += 10;
}

hobc_status check(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error(what, e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ULL; }
    return h;
}

}  // namespace

extern "C" {

hobc_status hobc_mlp_create(int n_in, int n_hidden, void* cuda_stream, hobc_mlp** out) {
    if (!out) return HOBC_ERR_ARG;
    *out = nullptr;
    if (n_in < 1 || n_in > 4096 || n_hidden < 1 || n_hidden > 4096) return HOBC_ERR_ARG;
    hobc_mlp_s* q = new hobc_mlp_s();
    q->nin = n_in;
    q->nh = n_hidden;
    q->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    q->P = ob3(q) + 1;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    alloc((void**)&q->params, q->P * sizeof(float));
    alloc((void**)&q->grads, q->P * sizeof(float));
    alloc((void**)&q->m, q->P * sizeof(float));
    alloc((void**)&q->v, q->P * sizeof(float));
    alloc((void**)&q->mean, n_in * sizeof(float));
    alloc((void**)&q->scale, n_in * sizeof(float));
    alloc((void**)&q->w1h, (size_t)n_hidden * n_in * sizeof(__nv_bfloat16));
    alloc((void**)&q->w2h, (size_t)n_hidden * n_hidden * sizeof(__nv_bfloat16));
    alloc((void**)&q->w3h, n_hidden * sizeof(__nv_bfloat16));
    alloc((void**)&q->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(q->params, 0, q->P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(q->m, 0, q->P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(q->v, 0, q->P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(q->mean, 0, n_in * sizeof(float));
    if (e == cudaSuccess) {
        std::vector<float> one(n_in, 1.f);
        e = cudaMemcpy(q->scale, one.data(), n_in * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        set_last_error("hobc_mlp_create", e);
        hobc_mlp_destroy(q);
        return HOBC_ERR_CUDA;
    }
    *out = q;
    return HOBC_OK;
}

void hobc_mlp_destroy(hobc_mlp* q) {
    if (!q) return;
    if (q->stream) cudaStreamSynchronize(q->stream);
    else cudaDeviceSynchronize();
    void* ps[] = {q->params, q->grads, q->m, q->v, q->mean, q->scale, q->w1h, q->w2h, q->w3h, q->loss,
                  q->xs, q->z1, q->h1, q->z2, q->h2, q->y, q->dy, q->dz2, q->dh1, q->dz1};
    for (void* p : ps) cudaFree(p);
    delete q;
}

int hobc_mlp_param_count(const hobc_mlp* q) { return q ? q->P : 0; }

hobc_status hobc_mlp_set_params(hobc_mlp* q, const float* host) {
    if (!q || !host) return HOBC_ERR_ARG;
    cudaError_t e = cudaMemcpy(q->params, host, q->P * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q->mean, host + q->P, q->nin * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q->scale, host + q->P + q->nin, q->nin * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(q->m, 0, q->P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(q->v, 0, q->P * sizeof(float));
    if (e != cudaSuccess) { set_last_error("hobc_mlp_set_params", e); return HOBC_ERR_CUDA; }
    q->step = 0;
    q->launches = 0;
    refresh_bf16(q);
    return check("hobc_mlp_set_params");
}

hobc_status hobc_mlp_get_params(const hobc_mlp* q, float* host) {
    if (!q || !host) return HOBC_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(q->stream);
    if (e == cudaSuccess) e = cudaMemcpy(host, q->params, q->P * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(host + q->P, q->mean, q->nin * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(host + q->P + q->nin, q->scale, q->nin * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_last_error("hobc_mlp_get_params", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

hobc_status hobc_mlp_forward(hobc_mlp* q, const float* x_dev, int batch, float* y_dev) {
    if (!q || !x_dev || !y_dev || batch < 1) return HOBC_ERR_ARG;
    cudaError_t e = ensure_capacity(q, batch);
    if (e != cudaSuccess) { set_last_error("hobc_mlp_forward", e); return HOBC_ERR_CUDA; }
    q->launches = 0;
    forward(q, x_dev, batch, y_dev);
    return check("hobc_mlp_forward");
}

hobc_status hobc_mlp_gradients(hobc_mlp* q, const float* x_dev, const float* t_dev, int batch, float* grad_dev,
                               float* loss_dev) {
    if (!q || !x_dev || !t_dev || batch < 1) return HOBC_ERR_ARG;
    cudaError_t e = ensure_capacity(q, batch);
    if (e != cudaSuccess) { set_last_error("hobc_mlp_gradients", e); return HOBC_ERR_CUDA; }
    q->launches = 0;
    forward(q, x_dev, batch, q->y);
    backward(q, t_dev, batch, loss_dev ? loss_dev : q->loss);
    if (grad_dev) {
        e = cudaMemcpyAsync(grad_dev, q->grads, q->P * sizeof(float), cudaMemcpyDeviceToDevice, q->stream);
        if (e != cudaSuccess) { set_last_error("hobc_mlp_gradients", e); return HOBC_ERR_CUDA; }
    }
    return check("hobc_mlp_gradients");
}

hobc_status hobc_mlp_train_step(hobc_mlp* q, const float* x_dev, const float* t_dev, int batch, float lr,
                                float weight_decay, float* loss_dev) {
    hobc_status s = hobc_mlp_gradients(q, x_dev, t_dev, batch, nullptr, loss_dev);
    if (s != HOBC_OK) return s;
    q->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)q->step), c2 = 1.f - powf(b2, (float)q->step);
    k_adamw<<<(q->P + 255) / 256, 256, 0, q->stream>>>(q->params, q->grads, q->m, q->v, q->P, lr, b1, b2, 1e-8f,
                                                       weight_decay, c1, c2);
    q->launches += 1;
    refresh_bf16(q);
    return check("hobc_mlp_train_step");
}

// Checkpoint: "HOBCMLP1", int32 nin, nh, step, P; float params[P], mean[nin],
// scale[nin], m[P], v[P]; uint64 FNV-1a checksum of everything before it.
hobc_status hobc_mlp_save(const hobc_mlp* q, const char* path) {
    if (!q || !path) return HOBC_ERR_ARG;
    const size_t P = q->P, nin = q->nin;
    std::vector<float> buf(3 * P + 2 * nin);
    cudaError_t e = cudaStreamSynchronize(q->stream);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data(), q->params, P * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + P, q->mean, nin * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + P + nin, q->scale, nin * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + P + 2 * nin, q->m, P * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + 2 * P + 2 * nin, q->v, P * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_last_error("hobc_mlp_save", e); return HOBC_ERR_CUDA; }
    const char magic[8] = {'H', 'O', 'B', 'C', 'M', 'L', 'P', '1'};
    const int32_t hdr[4] = {q->nin, q->nh, q->step, q->P};
    uint64_t h = 1469598103934665603ULL;
    h = fnv1a(magic, 8, h);
    h = fnv1a(hdr, sizeof(hdr), h);
    h = fnv1a(buf.data(), buf.size() * 4, h);
    FILE* f = fopen(path, "wb");
    if (!f) return HOBC_ERR_ARG;
    const bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
                    fwrite(buf.data(), 4, buf.size(), f) == buf.size() && fwrite(&h, 8, 1, f) == 1;
    fclose(f);
    return ok ? HOBC_OK : HOBC_ERR_ARG;
}

hobc_status hobc_mlp_load(hobc_mlp* q, const char* path) {
    if (!q || !path) return HOBC_ERR_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return HOBC_ERR_ARG;
    char magic[8];
    int32_t hdr[4];
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "HOBCMLP1", 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
              hdr[0] == q->nin && hdr[1] == q->nh && hdr[3] == q->P;
    std::vector<float> buf(3 * (size_t)q->P + 2 * (size_t)q->nin);
    uint64_t stored = 0;
    if (ok) ok = fread(buf.data(), 4, buf.size(), f) == buf.size() && fread(&stored, 8, 1, f) == 1;
    fclose(f);
    if (!ok) return HOBC_ERR_ARG;
    uint64_t h = 1469598103934665603ULL;
    h = fnv1a(magic, 8, h);
    h = fnv1a(hdr, sizeof(hdr), h);
    h = fnv1a(buf.data(), buf.size() * 4, h);
    if (h != stored) {
        set_last_error_text("hobc_mlp_load: checksum mismatch");
        return HOBC_ERR_ARG;
    }
    const size_t P = q->P, nin = q->nin;
    cudaError_t e = cudaMemcpy(q->params, buf.data(), P * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q->mean, buf.data() + P, nin * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q->scale, buf.data() + P + nin, nin * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q->m, buf.data() + P + 2 * nin, P * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q->v, buf.data() + 2 * P + 2 * nin, P * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { set_last_error("hobc_mlp_load", e); return HOBC_ERR_CUDA; }
    q->step = hdr[2];
    refresh_bf16(q);
    return check("hobc_mlp_load");
}

int hobc_mlp_last_launch_count(const hobc_mlp* q) { return q ? q->launches : 0; }

}  // extern "C"

// ================================================== features and learned path

namespace {

constexpr int kFeatChunk = 2048;     // spectral entries per features CTA

int bracket_size(const hobc_plan_s* p) { return 1 + std::min(kJL - 1, p->K); }   // the learned choice's J

cudaError_t ensure_learned_ws(hobc_plan_s* p) {
    if (p->log_grid) return cudaSuccess;
    const size_t B = (size_t)p->desc.batch;
    const size_t S = p->spec_elems;
    const size_t fch = (S + kFeatChunk - 1) / kFeatChunk;
    const size_t bch = (S + kBracketChunk - 1) / kBracketChunk;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(ptr, bytes); };
    if (p->nax == 2) {            // radial features (2D only)
        alloc((void**)&p->feat_partials, B * fch * 3 * kBins * sizeof(double));
        alloc((void**)&p->bin_tab, S);
    }
    alloc((void**)&p->feat, B * kFeat * sizeof(float));
    alloc((void**)&p->mlp_y, B * sizeof(float));
    alloc(&p->bracket_mu, B * kJL * p->esz);                 // kJL >= kJ slots serve every bracket scan
    alloc((void**)&p->mu_hat, B * sizeof(double));
    alloc((void**)&p->bracket_k0, B * sizeof(int));
    alloc((void**)&p->bracket_partials, B * bch * 2 * kJL * sizeof(double));
    alloc((void**)&p->bracket_G, B * kJL * sizeof(double));
    alloc((void**)&p->bracket_idx, B * sizeof(int));
    alloc((void**)&p->mu_val, B * sizeof(double));
    alloc((void**)&p->fell_back, B * sizeof(int));
    alloc((void**)&p->ahist_partials, B * ((S + kAChunk - 1) / kAChunk) * 3 * kABins * sizeof(double));
    alloc(&p->a_edges, (kABins + 1) * p->esz);
    alloc((void**)&p->k_hat, B * sizeof(int));
    alloc((void**)&p->refine_state, B * 4 * sizeof(double));
    alloc((void**)&p->log_grid, (size_t)p->K * sizeof(double));
    if (e == cudaSuccess) {       // the histogram's bin edges 10^(lo + b (hi - lo) / nb), in plan precision
        std::vector<double> ed(kABins + 1);
        for (int b = 0; b <= kABins; ++b) ed[b] = std::pow(10.0, kALo + (b * (kAHi - kALo)) / kABins);
        if (p->prec == HOBC_FP64) {
            e = cudaMemcpy(p->a_edges, ed.data(), ed.size() * sizeof(double), cudaMemcpyHostToDevice);
        } else {
            std::vector<float> ef(ed.begin(), ed.end());
            e = cudaMemcpy(p->a_edges, ef.data(), ef.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess && p->nax == 2) {
        GcvGeom geo;
        memset(&geo, 0, sizeof(geo));
        geo.ndim = 2; geo.fam = p->fam; geo.n0 = p->ax[0].n; geo.N0 = p->ax[0].N;
        geo.n1 = p->ax[1].n; geo.N1 = p->ax[1].N; geo.W1 = p->ax[1].W;
        geo.S = (long long)S;
        k_bin_table<<<(unsigned)std::min<size_t>((S + 255) / 256, 4096), 256, 0, p->stream>>>(
            geo, p->fam == HOBC_FAMILY_FOURIER, p->bin_tab);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {       // once per plan: the grid's logarithms and order, on the host
        std::vector<double> grid(p->K), lg(p->K);
        e = cudaMemcpy(grid.data(), p->mu, p->K * sizeof(double), cudaMemcpyDeviceToHost);
        p->grid_ascending = 1;
        for (int k = 0; k < p->K; ++k) {
            lg[k] = std::log10(grid[k]);
            if (k > 0 && !(grid[k] > grid[k - 1])) p->grid_ascending = 0;
        }
        if (e == cudaSuccess) e = cudaMemcpy(p->log_grid, lg.data(), p->K * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) free_learned_ws(p);
    return e;
}

template <typename T>
hobc_status run_features(hobc_plan_s* p, const void* ghat, const void* D, float* X) {
    const long long S = (long long)p->spec_elems;
    const int nch = (int)((S + kFeatChunk - 1) / kFeatChunk);
    const unsigned grid = (unsigned)(nch * (long long)p->desc.batch);
    if (p->fam == HOBC_FAMILY_FOURIER)
        k_features<T, true><<<grid, 256, 0, p->stream>>>(reinterpret_cast<const C2<T>*>(ghat),
                                                         reinterpret_cast<const C2<T>*>(D), S, p->desc.psf_per_item,
                                                         S, kFeatChunk, p->bin_tab, p->feat_partials);
    else
        k_features<T, false><<<grid, 256, 0, p->stream>>>(reinterpret_cast<const T*>(ghat),
                                                          reinterpret_cast<const T*>(D), S, p->desc.psf_per_item,
                                                          S, kFeatChunk, p->bin_tab, p->feat_partials);
    k_features_finalize<<<p->desc.batch, 64, 0, p->stream>>>(p->feat_partials, nch, X);
    p->launches += 2;
    return check("hobc_features");
}

// Histogram features: the binned choice's histogram over log10 a, then
// k_hist_features.
template <typename T>
hobc_status run_features_hist(hobc_plan_s* p, const void* ghat, const void* D, float* X) {
    const int B = p->desc.batch;
    GcvGeom geo;
    memset(&geo, 0, sizeof(geo));
    const AxisHost& last = p->ax[p->nax - 1];
    geo.ndim = p->nax; geo.fam = p->fam; geo.n0 = p->ax[0].n; geo.N0 = p->ax[0].N;
    geo.n1 = last.n; geo.N1 = last.N; geo.W1 = last.W; geo.lap = p->desc.L == HOBC_L_LAPLACIAN;
    geo.S = (long long)p->spec_elems;
    geo.chunk = kAChunk;
    const int nch = (int)((geo.S + kAChunk - 1) / kAChunk);
    const unsigned gridA = (unsigned)(nch * (long long)B);
    const T* edges = reinterpret_cast<const T*>(p->a_edges);
    if (p->fam == HOBC_FAMILY_FOURIER)
        k_ahist<T, true><<<gridA, 256, 0, p->stream>>>(reinterpret_cast<const C2<T>*>(ghat),
                                                        reinterpret_cast<const C2<T>*>(D), geo.S, p->desc.psf_per_item,
                                                        geo, edges, p->ahist_partials);
    else
        k_ahist<T, false><<<gridA, 256, 0, p->stream>>>(reinterpret_cast<const T*>(ghat),
                                                         reinterpret_cast<const T*>(D), geo.S, p->desc.psf_per_item,
                                                         geo, edges, p->ahist_partials);
    k_hist_features<<<B, kABins, 0, p->stream>>>(p->ahist_partials, nch, X);
    p->launches += 2;
    return check("hobc_features_hist");
}

template <typename T>
hobc_status run_learned(hobc_plan_s* p, hobc_mlp_s* q, const void* g, const void* psf, void* f, double* mu_out,
                        int* fb_out) {
    const int B = p->desc.batch, K = p->K;
    const int J = bracket_size(p);
    hobc_status s = run_eig<T>(p, psf, p->D);
    if (s == HOBC_OK) s = run_analysis<T>(p, g, p->G);
    if (s == HOBC_OK)
        s = q->feature_kind == HOBC_FEATURES_HIST ? run_features_hist<T>(p, p->G, p->D, p->feat)
                                                  : run_features<T>(p, p->G, p->D, p->feat);
    if (s != HOBC_OK) return s;
    cudaError_t e = ensure_capacity(q, B);
    if (e != cudaSuccess) { set_last_error("hobc_deblur_learned", e); return HOBC_ERR_CUDA; }
    const cudaStream_t own = q->stream;
    q->stream = p->stream;
    forward(q, p->feat, B, p->mlp_y);
    q->stream = own;
    p->launches += 6;
    T* lists = reinterpret_cast<T*>(p->bracket_mu);
    k_bracket_setup<T, kJL><<<(B + 127) / 128, 128, 0, p->stream>>>(p->mlp_y, p->mu, p->log_grid, K, J, lists, p->mu_hat,
                                                                p->bracket_k0, B);
    // G at the bracket values
    GcvGeom geo;
    memset(&geo, 0, sizeof(geo));
    const AxisHost& last = p->ax[p->nax - 1];
    geo.ndim = p->nax; geo.fam = p->fam; geo.n0 = p->ax[0].n; geo.N0 = p->ax[0].N;
    geo.n1 = last.n; geo.N1 = last.N; geo.W1 = last.W; geo.lap = p->desc.L == HOBC_L_LAPLACIAN;
    geo.S = (long long)p->spec_elems;
    geo.K = kJL;
    geo.chunk = kBracketChunk;
    const int nchJ = (int)((geo.S + kBracketChunk - 1) / kBracketChunk);
    const unsigned gridJ = (unsigned)(nchJ * (long long)B);
    if (p->fam == HOBC_FAMILY_FOURIER)
        k_gcv_bracket<T, true, kJL><<<gridJ, 256, 0, p->stream>>>(
            reinterpret_cast<const C2<T>*>(p->G), reinterpret_cast<const C2<T>*>(p->D), (long long)p->spec_elems,
            p->desc.psf_per_item, lists, geo, p->bracket_partials);
    else
        k_gcv_bracket<T, false, kJL><<<gridJ, 256, 0, p->stream>>>(
            reinterpret_cast<const T*>(p->G), reinterpret_cast<const T*>(p->D), (long long)p->spec_elems,
            p->desc.psf_per_item, lists, geo, p->bracket_partials);
    k_bracket_finalize<kJL><<<B, 256, 0, p->stream>>>(p->bracket_partials, nchJ, p->bracket_G);
    double* mu_val = mu_out ? mu_out : p->mu_val;
    int* fb = fb_out ? fb_out : p->fell_back;
    k_bracket_decide<<<(B + 127) / 128, 128, 0, p->stream>>>(p->bracket_G, J, kJL, p->bracket_k0, K, p->mu_hat, mu_val, fb, B);
    // the full scan, only for the problems that fell back
    geo.K = K;
    geo.chunk = p->gcv_chunk;
    const size_t smemK = 4 * (size_t)geo.chunk * sizeof(T);
    const unsigned gridK = (unsigned)(p->gcv_chunks * (long long)B);
    if (p->fam == HOBC_FAMILY_FOURIER)
        k_gcv_masked<T, true><<<gridK, 256, smemK, p->stream>>>(
            reinterpret_cast<const C2<T>*>(p->G), reinterpret_cast<const C2<T>*>(p->D), (long long)p->spec_elems,
            p->desc.psf_per_item, reinterpret_cast<const T*>(p->muT), geo, fb, p->partials);
    else
        k_gcv_masked<T, false><<<gridK, 256, smemK, p->stream>>>(
            reinterpret_cast<const T*>(p->G), reinterpret_cast<const T*>(p->D), (long long)p->spec_elems,
            p->desc.psf_per_item, reinterpret_cast<const T*>(p->muT), geo, fb, p->partials);
    k_masked_finalize<<<B, 256, 0, p->stream>>>(p->partials, p->gcv_chunks, K, fb, p->mu, mu_val, nullptr);
    p->launches += 6;
    s = check("hobc_deblur_learned");
    if (s != HOBC_OK) return s;
    return run_filter_synthesis_mu<T>(p, p->G, p->D, mu_val, f);
}

template <typename T>
GcvGeom spectrum_geo(const hobc_plan_s* p) {
    GcvGeom geo;
    memset(&geo, 0, sizeof(geo));
    const AxisHost& last = p->ax[p->nax - 1];
    geo.ndim = p->nax; geo.fam = p->fam; geo.n0 = p->ax[0].n; geo.N0 = p->ax[0].N;
    geo.n1 = last.n; geo.N1 = last.N; geo.W1 = last.W; geo.lap = p->desc.L == HOBC_L_LAPLACIAN;
    geo.S = (long long)p->spec_elems;
    return geo;
}

// The binned choice on a plan's spectra: histogram, k_hat, exact G on the
// bracket, decision, and the masked full scan for the problems that fell back.
template <typename T>
hobc_status run_gcv_binned(hobc_plan_s* p, const void* ghat, const void* D, int* mu_idx, int* fb, int* khat) {
    const int B = p->desc.batch, K = p->K;
    const bool cplx = p->fam == HOBC_FAMILY_FOURIER;
    typedef C2<T> CT;
    GcvGeom geo = spectrum_geo<T>(p);
    geo.chunk = kAChunk;
    const int nch = (int)((geo.S + kAChunk - 1) / kAChunk);
    const unsigned gridA = (unsigned)(nch * (long long)B);
    const T* edges = reinterpret_cast<const T*>(p->a_edges);
    if (cplx)
        k_ahist<T, true><<<gridA, 256, 0, p->stream>>>(reinterpret_cast<const CT*>(ghat), reinterpret_cast<const CT*>(D),
                                                        geo.S, p->desc.psf_per_item, geo, edges, p->ahist_partials);
    else
        k_ahist<T, false><<<gridA, 256, 0, p->stream>>>(reinterpret_cast<const T*>(ghat), reinterpret_cast<const T*>(D),
                                                         geo.S, p->desc.psf_per_item, geo, edges, p->ahist_partials);
    T* lists = reinterpret_cast<T*>(p->bracket_mu);
    k_binned_khat<T><<<B, 256, 0, p->stream>>>(p->ahist_partials, nch, p->mu, K, khat, p->bracket_k0, lists);
    geo.K = kJ;
    geo.chunk = kBracketChunk;
    const int nchJ = (int)((geo.S + kBracketChunk - 1) / kBracketChunk);
    const unsigned gridJ = (unsigned)(nchJ * (long long)B);
    if (cplx)
        k_gcv_bracket<T, true><<<gridJ, 256, 0, p->stream>>>(reinterpret_cast<const CT*>(ghat),
                                                              reinterpret_cast<const CT*>(D), geo.S,
                                                              p->desc.psf_per_item, lists, geo, p->bracket_partials);
    else
        k_gcv_bracket<T, false><<<gridJ, 256, 0, p->stream>>>(reinterpret_cast<const T*>(ghat),
                                                               reinterpret_cast<const T*>(D), geo.S,
                                                               p->desc.psf_per_item, lists, geo, p->bracket_partials);
    k_bracket_finalize<<<B, 256, 0, p->stream>>>(p->bracket_partials, nchJ, p->bracket_G);
    k_binned_decide<<<(B + 127) / 128, 128, 0, p->stream>>>(p->bracket_G, K, p->bracket_k0, mu_idx, fb, B);
    geo.K = K;
    geo.chunk = p->gcv_chunk;
    const size_t smemK = 4 * (size_t)geo.chunk * sizeof(T);
    const unsigned gridK = (unsigned)(p->gcv_chunks * (long long)B);
    if (cplx)
        k_gcv_masked<T, true><<<gridK, 256, smemK, p->stream>>>(
            reinterpret_cast<const CT*>(ghat), reinterpret_cast<const CT*>(D), geo.S, p->desc.psf_per_item,
            reinterpret_cast<const T*>(p->muT), geo, fb, p->partials);
    else
        k_gcv_masked<T, false><<<gridK, 256, smemK, p->stream>>>(
            reinterpret_cast<const T*>(ghat), reinterpret_cast<const T*>(D), geo.S, p->desc.psf_per_item,
            reinterpret_cast<const T*>(p->muT), geo, fb, p->partials);
    k_masked_finalize<<<B, 256, 0, p->stream>>>(p->partials, p->gcv_chunks, K, fb, p->mu, nullptr, mu_idx);
    p->launches += 8;
    return check("hobc_gcv_binned");
}

// The refinement on a plan's spectra from the grid argmin mu_idx: one init
// launch, then per round the bracket scan, its finalize and the step.
template <typename T>
hobc_status run_gcv_refine(hobc_plan_s* p, const void* ghat, const void* D, const int* mu_idx, double* mu_out,
                           double* G_out) {
    const int B = p->desc.batch, K = p->K;
    const bool cplx = p->fam == HOBC_FAMILY_FOURIER;
    typedef C2<T> CT;
    T* lists = reinterpret_cast<T*>(p->bracket_mu);
    const unsigned gridB = (unsigned)((B + 127) / 128);
    k_refine_init<T><<<gridB, 128, 0, p->stream>>>(mu_idx, p->mu, p->log_grid, K, p->refine_state, lists, B);
    GcvGeom geo = spectrum_geo<T>(p);
    geo.K = kJ;
    geo.chunk = kBracketChunk;
    const int nchJ = (int)((geo.S + kBracketChunk - 1) / kBracketChunk);
    const unsigned gridJ = (unsigned)(nchJ * (long long)B);
    for (int r = 0; r < kRefineRounds; ++r) {
        if (cplx)
            k_gcv_bracket<T, true><<<gridJ, 256, 0, p->stream>>>(reinterpret_cast<const CT*>(ghat),
                                                                  reinterpret_cast<const CT*>(D), geo.S,
                                                                  p->desc.psf_per_item, lists, geo,
                                                                  p->bracket_partials);
        else
            k_gcv_bracket<T, false><<<gridJ, 256, 0, p->stream>>>(reinterpret_cast<const T*>(ghat),
                                                                   reinterpret_cast<const T*>(D), geo.S,
                                                                   p->desc.psf_per_item, lists, geo,
                                                                   p->bracket_partials);
        k_bracket_finalize<<<B, 256, 0, p->stream>>>(p->bracket_partials, nchJ, p->bracket_G);
        k_refine_step<T><<<gridB, 128, 0, p->stream>>>(p->bracket_G, p->refine_state, lists,
                                                        r == kRefineRounds - 1, mu_out, G_out, B);
    }
    p->launches += 1 + 3 * kRefineRounds;
    return check("hobc_gcv_refine");
}

template <typename T>
hobc_status run_deblur_refined(hobc_plan_s* p, const void* g, const void* psf, void* f, int* mu_idx,
                               double* mu_out) {
    hobc_status s = run_eig<T>(p, psf, p->D);
    if (s == HOBC_OK) s = run_analysis<T>(p, g, p->G);
    if (s == HOBC_OK) s = run_gcv<T>(p, p->G, p->D, nullptr, mu_idx);
    if (s == HOBC_OK) s = run_gcv_refine<T>(p, p->G, p->D, mu_idx, mu_out, nullptr);
    if (s == HOBC_OK) s = run_filter_synthesis_mu<T>(p, p->G, p->D, mu_out, f);
    return s;
}

template <typename T>
hobc_status run_deblur_binned(hobc_plan_s* p, const void* g, const void* psf, void* f, int* mu_idx, int* fb) {
    hobc_status s = run_eig<T>(p, psf, p->D);
    if (s == HOBC_OK) s = run_analysis<T>(p, g, p->G);
    if (s == HOBC_OK) s = run_gcv_binned<T>(p, p->G, p->D, mu_idx, fb, p->k_hat);
    if (s == HOBC_OK) s = run_filter_synthesis<T>(p, p->G, p->D, mu_idx, f);
    return s;
}

}  // namespace

extern "C" {

hobc_status hobc_features(hobc_plan* p, const void* ghat_dev, const void* d_dev, float* x_dev) {
    if (!p || !ghat_dev || !d_dev || !x_dev) return HOBC_ERR_ARG;
    if (p->nax != 2 || p->fam == HOBC_FAMILY_REFLECTIVE || p->fam == HOBC_FAMILY_PERIODIC || plain_only_family(p->fam))
        return HOBC_ERR_UNSUPPORTED;
    cudaError_t e = ensure_learned_ws(p);
    if (e != cudaSuccess) { set_last_error("hobc_features", e); return HOBC_ERR_CUDA; }
    p->launches = 0;
    return p->prec == HOBC_FP64 ? run_features<double>(p, ghat_dev, d_dev, x_dev)
                                : run_features<float>(p, ghat_dev, d_dev, x_dev);
}

hobc_status hobc_features_hist(hobc_plan* p, const void* ghat_dev, const void* d_dev, float* x_dev) {
    if (!p || !ghat_dev || !d_dev || !x_dev) return HOBC_ERR_ARG;
    if (p->fam == HOBC_FAMILY_REFLECTIVE || p->fam == HOBC_FAMILY_PERIODIC || plain_only_family(p->fam))
        return HOBC_ERR_UNSUPPORTED;
    cudaError_t e = ensure_learned_ws(p);
    if (e != cudaSuccess) { set_last_error("hobc_features_hist", e); return HOBC_ERR_CUDA; }
    p->launches = 0;
    return p->prec == HOBC_FP64 ? run_features_hist<double>(p, ghat_dev, d_dev, x_dev)
                                : run_features_hist<float>(p, ghat_dev, d_dev, x_dev);
}

hobc_status hobc_mlp_fit_scaling(hobc_mlp* q, const float* x_dev, int rows) {
    if (!q || !x_dev || rows < 1) return HOBC_ERR_ARG;
    k_fit_scaling<<<q->nin, 256, 0, q->stream>>>(x_dev, rows, q->nin, q->mean, q->scale);
    q->launches = 1;
    return check("hobc_mlp_fit_scaling");
}

hobc_status hobc_mlp_set_feature_kind(hobc_mlp* q, int kind) {
    if (!q || (kind != HOBC_FEATURES_RADIAL && kind != HOBC_FEATURES_HIST)) return HOBC_ERR_ARG;
    q->feature_kind = kind;
    return HOBC_OK;
}

int hobc_mlp_feature_kind(const hobc_mlp* q) { return q ? q->feature_kind : -1; }

hobc_status hobc_deblur_learned(hobc_plan* p, hobc_mlp* q, const void* g_dev, const void* psf_dev, void* f_dev,
                                double* mu_dev, int* fell_back_dev) {
    if (!p || !q || !g_dev || !psf_dev || !f_dev) return HOBC_ERR_ARG;
    if ((p->nax != 2 && q->feature_kind == HOBC_FEATURES_RADIAL) || q->nin != kFeat ||
        p->fam == HOBC_FAMILY_REFLECTIVE || p->fam == HOBC_FAMILY_PERIODIC || plain_only_family(p->fam))
        return HOBC_ERR_UNSUPPORTED;
    cudaError_t e = ensure_learned_ws(p);
    if (e != cudaSuccess) { set_last_error("hobc_deblur_learned", e); return HOBC_ERR_CUDA; }
    if (!p->grid_ascending) {
        set_last_error_text("hobc_deblur_learned: the mu grid must be strictly increasing");
        return HOBC_ERR_ARG;
    }
    p->launches = 0;
    return p->prec == HOBC_FP64 ? run_learned<double>(p, q, g_dev, psf_dev, f_dev, mu_dev, fell_back_dev)
                                : run_learned<float>(p, q, g_dev, psf_dev, f_dev, mu_dev, fell_back_dev);
}

hobc_status hobc_gcv_binned(hobc_plan* p, const void* ghat_dev, const void* d_dev, int* mu_index_dev,
                            int* fell_back_dev, int* k_hat_dev) {
    if (!p || !ghat_dev || !d_dev || !mu_index_dev) return HOBC_ERR_ARG;
    if (plain_only_family(p->fam)) return HOBC_ERR_UNSUPPORTED;
    cudaError_t e = ensure_learned_ws(p);
    if (e != cudaSuccess) { set_last_error("hobc_gcv_binned", e); return HOBC_ERR_CUDA; }
    if (!p->grid_ascending) {
        set_last_error_text("hobc_gcv_binned: the mu grid must be strictly increasing");
        return HOBC_ERR_ARG;
    }
    p->launches = 0;
    int* fb = fell_back_dev ? fell_back_dev : p->fell_back;
    int* kh = k_hat_dev ? k_hat_dev : p->k_hat;
    return p->prec == HOBC_FP64 ? run_gcv_binned<double>(p, ghat_dev, d_dev, mu_index_dev, fb, kh)
                                : run_gcv_binned<float>(p, ghat_dev, d_dev, mu_index_dev, fb, kh);
}

hobc_status hobc_deblur_binned(hobc_plan* p, const void* g_dev, const void* psf_dev, void* f_dev, int* mu_index_dev,
                               int* fell_back_dev) {
    if (!p || !g_dev || !psf_dev || !f_dev) return HOBC_ERR_ARG;
    if (plain_only_family(p->fam)) return HOBC_ERR_UNSUPPORTED;
    cudaError_t e = ensure_learned_ws(p);
    if (e != cudaSuccess) { set_last_error("hobc_deblur_binned", e); return HOBC_ERR_CUDA; }
    if (!p->grid_ascending) {
        set_last_error_text("hobc_deblur_binned: the mu grid must be strictly increasing");
        return HOBC_ERR_ARG;
    }
    p->launches = 0;
    int* mi = mu_index_dev ? mu_index_dev : p->mu_idx;
    int* fb = fell_back_dev ? fell_back_dev : p->fell_back;
    return p->prec == HOBC_FP64 ? run_deblur_binned<double>(p, g_dev, psf_dev, f_dev, mi, fb)
                                : run_deblur_binned<float>(p, g_dev, psf_dev, f_dev, mi, fb);
}

hobc_status hobc_gcv_refine(hobc_plan* p, const void* ghat_dev, const void* d_dev, const int* mu_index_dev,
                            double* mu_dev, double* gcv_dev) {
    if (!p || !ghat_dev || !d_dev || !mu_index_dev || !mu_dev) return HOBC_ERR_ARG;
    if (plain_only_family(p->fam)) return HOBC_ERR_UNSUPPORTED;
    cudaError_t e = ensure_learned_ws(p);
    if (e != cudaSuccess) { set_last_error("hobc_gcv_refine", e); return HOBC_ERR_CUDA; }
    if (!p->grid_ascending) {
        set_last_error_text("hobc_gcv_refine: the mu grid must be strictly increasing");
        return HOBC_ERR_ARG;
    }
    p->launches = 0;
    return p->prec == HOBC_FP64 ? run_gcv_refine<double>(p, ghat_dev, d_dev, mu_index_dev, mu_dev, gcv_dev)
                                : run_gcv_refine<float>(p, ghat_dev, d_dev, mu_index_dev, mu_dev, gcv_dev);
}

hobc_status hobc_filter_synthesis_mu(hobc_plan* p, const void* ghat_dev, const void* d_dev, const double* mu_dev,
                                     void* f_dev) {
    if (!p || !ghat_dev || !d_dev || !mu_dev || !f_dev) return HOBC_ERR_ARG;
    p->launches = 0;
    hobc_status s = p->prec == HOBC_FP64 ? run_filter_synthesis_mu<double>(p, ghat_dev, d_dev, mu_dev, f_dev)
                                         : run_filter_synthesis_mu<float>(p, ghat_dev, d_dev, mu_dev, f_dev);
    return s == HOBC_OK ? check("hobc_filter_synthesis_mu") : s;
}

hobc_status hobc_deblur_refined(hobc_plan* p, const void* g_dev, const void* psf_dev, void* f_dev, int* mu_index_dev,
                                double* mu_dev) {
    if (!p || !g_dev || !psf_dev || !f_dev) return HOBC_ERR_ARG;
    if (plain_only_family(p->fam)) return HOBC_ERR_UNSUPPORTED;
    cudaError_t e = ensure_learned_ws(p);
    if (e != cudaSuccess) { set_last_error("hobc_deblur_refined", e); return HOBC_ERR_CUDA; }
    if (!p->grid_ascending) {
        set_last_error_text("hobc_deblur_refined: the mu grid must be strictly increasing");
        return HOBC_ERR_ARG;
    }
    p->launches = 0;
    int* mi = mu_index_dev ? mu_index_dev : p->mu_idx;
    double* mu = mu_dev ? mu_dev : p->mu_val;
    return p->prec == HOBC_FP64 ? run_deblur_refined<double>(p, g_dev, psf_dev, f_dev, mi, mu)
                                : run_deblur_refined<float>(p, g_dev, psf_dev, f_dev, mi, mu);
}

}  // extern "C"
