// The exact GCV functional of Eq. (eq:gcv) for the real families
// (include/hobc_exact.h).  Per plan, once: T_a of each axis from the FP64
// synthesis of the identity, split by rows on the host (FP64): the interior
// rows are X_a^T W_a with X_a^T orthonormal and W_a = [bhat_L | I | bhat_R],
// the 2k extension rows (at the border indices) are V_a.  Then
//   ||T_0 P T_1^T||^2 = ||W0 P W1^T||^2 + ||V0 P W1^T||^2 + ||W0 P V1^T||^2
//                       + ||V0 P V1^T||^2,
// every term a sum of squares (no cancellation between large terms, which
// the Gram form |P|^2 + P^T (T^T T - I) P suffers: T_C at n = 1024 has
// condition ~2e4).  Per call: one CTA per spectral column, one per spectral
// row, an FP64 reduction and the argmin; 1D plans one CTA per problem.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/hobc_exact.h"
#include "hobc_internal.h"
#include "hobc_kernels.cuh"

struct hobc_exact_s {
    int k;                 // border vectors per side (1: sine and cosine, 2: degree 3, 0: orthogonal T)
    int N[2];              // interior length n_a - 2k
    int bidx[2][4];        // border indices of each axis: 0..k-1, n-k..n-1
    void* bhat[2];         // [2k][N_a] plan precision: X_a times the interior part of each border column
    void* V[2];            // [2k][n_a] plan precision: the extension rows of T_a
    double* Vd[2];         // [2k][n_a] FP64 copy of V_a (the V_0 P V_1^T term)
    void* col_out;         // [batch][n_1][3 + 2k][K]: |W0 P W1^T col|^2, |V0 P W1^T col|^2, sum sigma, V0 P col
    void* row_out;         // [batch][n_0][K]: |W0 P V1^T row|^2
    double* G;             // [batch][K] when the caller passes no curve
};

namespace hobc {

constexpr int kExKMax = 2;             // border vectors per side at most (degree 3)
constexpr int kExB = 2 * kExKMax;
constexpr int kExSlots = 8;            // reduction: line slices per grid value

namespace {

// Column t of T_X of one axis (T[i * n + t]) from the FP64 synthesis of e_t.
hobc_status axis_matrix(int fam, int n, cudaStream_t st, std::vector<double>& T) {
    hobc_plan_desc q;
    memset(&q, 0, sizeof(q));
    q.ndim = 1; q.n[0] = n; q.psf[0] = 1; q.family = (hobc_family)fam; q.psf_symmetric = 1;
    q.bc_degree = fam == HOBC_FAMILY_SINE ? 1 : (fam == HOBC_FAMILY_COSINE ? 2 : 3);
    q.L = HOBC_L_IDENTITY; q.prec = HOBC_FP64; q.n_mu = 1; q.batch = n; q.psf_per_item = 0;
    const double one = 1.0;
    hobc_plan* ip = nullptr;
    hobc_status s = hobc_plan_create(&q, &one, st, &ip);
    if (s != HOBC_OK) return s;
    double *I = nullptr, *out = nullptr;
    cudaError_t e = cudaMalloc((void**)&I, (size_t)n * n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&out, (size_t)n * n * sizeof(double));
    std::vector<double> eye((size_t)n * n, 0.0), Y((size_t)n * n);
    for (int i = 0; i < n; ++i) eye[(size_t)i * n + i] = 1.0;
    if (e == cudaSuccess) e = cudaMemcpy(I, eye.data(), eye.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) s = hobc_synthesis(ip, I, out);
    if (e == cudaSuccess && s == HOBC_OK) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && s == HOBC_OK) e = cudaMemcpy(Y.data(), out, Y.size() * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(I);
    cudaFree(out);
    hobc_plan_destroy(ip);
    if (s != HOBC_OK) return s;
    if (e != cudaSuccess) { set_last_error("hobc_gcv_exact (transform matrix)", e); return HOBC_ERR_CUDA; }
    T.assign((size_t)n * n, 0.0);
    for (int t = 0; t < n; ++t)                 // row t of the output is T e_t
        for (int i = 0; i < n; ++i) T[(size_t)i * n + t] = Y[(size_t)t * n + i];
    return HOBC_OK;
}

// The row split of T (k border indices per side): interior rows k..n-k-1 are
// X^T [bhat_L | I | bhat_R] with X^T = T[interior][interior] orthonormal, and
// the extension rows (the border indices) are V.  Checks the orthonormality.
hobc_status split_rows(const std::vector<double>& T, int n, int k, std::vector<double>& bhat, std::vector<double>& V) {
    const int N = n - 2 * k;
    double dev = 0;
    for (int i = 0; i < N; ++i)                 // rows of X^T: X^T X = I
        for (int j = i; j < N; ++j) {
            double acc = 0;
            for (int m = 0; m < N; ++m) acc += T[(size_t)(k + i) * n + k + m] * T[(size_t)(k + j) * n + k + m];
            dev = std::max(dev, std::fabs(acc - (i == j ? 1.0 : 0.0)));
        }
    if (dev > 1e-10) {
        set_last_error_text("hobc_gcv_exact: the interior block of T is not orthonormal");
        return HOBC_ERR_UNSUPPORTED;
    }
    bhat.assign((size_t)std::max(2 * k * N, 1), 0.0);
    V.assign((size_t)std::max(2 * k * n, 1), 0.0);
    for (int b = 0; b < 2 * k; ++b) {
        const int col = b < k ? b : n - 2 * k + b;
        for (int i = 0; i < N; ++i) {           // (X t_int)[i] = sum_m X^T[m][i] T[k + m][col]
            double acc = 0;
            for (int m = 0; m < N; ++m) acc += T[(size_t)(k + m) * n + k + i] * T[(size_t)(k + m) * n + col];
            bhat[(size_t)b * N + i] = acc;
        }
        for (int a = 0; a < n; ++a) V[(size_t)b * n + a] = T[(size_t)col * n + a];
    }
    return HOBC_OK;
}

template <typename T> cudaError_t upload(void** dst, const std::vector<double>& v) {
    std::vector<T> w(v.begin(), v.end());
    cudaError_t e = cudaMalloc(dst, w.size() * sizeof(T));
    if (e == cudaSuccess) e = cudaMemcpy(*dst, w.data(), w.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

GcvGeom exact_geo(const hobc_plan_s* p) {
    GcvGeom geo;
    memset(&geo, 0, sizeof(geo));
    const AxisHost& last = p->ax[p->nax - 1];
    geo.ndim = p->nax; geo.fam = p->fam; geo.n0 = p->ax[0].n; geo.N0 = p->ax[0].N;
    geo.n1 = last.n; geo.N1 = last.N; geo.W1 = last.W; geo.lap = p->desc.L == HOBC_L_LAPLACIAN;
    geo.S = (long long)p->spec_elems;
    geo.K = p->K;
    return geo;
}

struct ExAxis {            // one axis's split, as the kernels see it
    const void* bhat;
    const void* V;
    int n, N;
    int bidx[kExB];
};

}  // namespace

// a and ghat of stored entry e into shared memory: entries with s = 0 carry
// a = inf (sigma = 0, so they drop out as in the approximation).
template <typename T>
__device__ __forceinline__ void ex_stage(const T* sp, const T* dp, const GcvGeom& geo, long long e, T& a, T& g) {
    const typename Pack4<T>::t v = gcv_term<T, false>(sp[e], dp[e], geo, e);
    const bool live = v.z > (T)0;
    a = live ? v.x : (T)INFINITY;
    g = live ? sp[e] : (T)0;
}

// 2D, one CTA per spectral column c (entries c n0 + a), one grid value per
// thread.  Also stages the border columns.  For an interior column j = c - k:
//   ww = sum_i (W0 P W1^T)[i][j]^2,  vw = sum_r (V0 P W1^T)[r][j]^2;
// for every column: den = sum sigma and the projections (V0 P)[r][c].
// grid = (n1, items), block = 256; dynamic shared memory 2 (1 + 2k) n0 sizeof(T).
template <typename T>
__global__ void __launch_bounds__(256)
k_ex_cols(const T* __restrict__ spec, const T* __restrict__ D, long long d_psf_stride, int psf_per,
          const T* __restrict__ muT, GcvGeom geo, ExAxis A0, ExAxis A1, int k, T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n0 = A0.n, n1 = A1.n, nb = 2 * k;
    T* sa = reinterpret_cast<T*>(smem_raw);     // [1 + nb][n0]
    T* sg = sa + (size_t)(1 + nb) * n0;
    const int c = blockIdx.x;
    const long long item = blockIdx.y;
    const T* sp = spec + item * geo.S;
    const T* dp = D + (psf_per ? item : 0) * d_psf_stride;
    for (int s = 0; s <= nb; ++s) {
        const int col = s == 0 ? c : A1.bidx[s - 1];
        for (int a = threadIdx.x; a < n0; a += blockDim.x)
            ex_stage<T>(sp, dp, geo, (long long)col * n0 + a, sa[s * n0 + a], sg[s * n0 + a]);
    }
    __syncthreads();
    const T* b0 = reinterpret_cast<const T*>(A0.bhat);
    const T* b1 = reinterpret_cast<const T*>(A1.bhat);
    const T* V0 = reinterpret_cast<const T*>(A0.V);
    const bool inter = c >= k && c < n1 - k;
    const int jj = c - k;
    T beta[kExB];
#pragma unroll
    for (int bl = 0; bl < kExB; ++bl) beta[bl] = (inter && bl < nb) ? b1[(size_t)bl * A1.N + jj] : (T)0;
    const int K = geo.K;
    const int nval = 3 + nb;
    T* o = out + (item * n1 + c) * (long long)nval * K;
    for (int jb = 0; jb < K; jb += blockDim.x) {
        const int j = jb + threadIdx.x;
        const T mu = j < K ? muT[j] : (T)1;
        T gam[kExB];                            // P[bk][c] + sum_bl P[bk][bl] bhat1[bl][jj]
#pragma unroll
        for (int bk = 0; bk < kExB; ++bk) {
            gam[bk] = 0;
            if (bk < nb) {
                const int ar = A0.bidx[bk];
                T gv = pair_rcp(sa[ar] + mu) * sg[ar];
#pragma unroll
                for (int bl = 0; bl < kExB; ++bl)
                    if (bl < nb) gv += pair_rcp(sa[(1 + bl) * n0 + ar] + mu) * sg[(1 + bl) * n0 + ar] * beta[bl];
                gam[bk] = gv;
            }
        }
        T ww = 0, den = 0, s[kExB], sb[kExB][kExB];
#pragma unroll
        for (int r = 0; r < kExB; ++r) {
            s[r] = 0;
#pragma unroll
            for (int bl = 0; bl < kExB; ++bl) sb[r][bl] = 0;
        }
        for (int a = 0; a < n0; ++a) {
            const T s0 = pair_rcp(sa[a] + mu);
            const T P0 = s0 * sg[a];
            den += s0;
            T Pb[kExB];
#pragma unroll
            for (int bl = 0; bl < kExB; ++bl)
                Pb[bl] = bl < nb ? pair_rcp(sa[(1 + bl) * n0 + a] + mu) * sg[(1 + bl) * n0 + a] : (T)0;
#pragma unroll
            for (int r = 0; r < kExB; ++r)
                if (r < nb) {
                    const T v = __ldg(V0 + (size_t)r * n0 + a);
                    s[r] += v * P0;
#pragma unroll
                    for (int bl = 0; bl < kExB; ++bl)
                        if (bl < nb) sb[r][bl] += v * Pb[bl];
                }
            if (inter && a >= k && a < n0 - k) {
                const int i = a - k;
                T w = P0;
#pragma unroll
                for (int bl = 0; bl < kExB; ++bl)
                    if (bl < nb) w += Pb[bl] * beta[bl];
#pragma unroll
                for (int bk = 0; bk < kExB; ++bk)
                    if (bk < nb) w += __ldg(b0 + (size_t)bk * A0.N + i) * gam[bk];
                ww += w * w;
            }
        }
        T vw = 0;
        if (inter)
#pragma unroll
            for (int r = 0; r < kExB; ++r)
                if (r < nb) {
                    T v = s[r];
#pragma unroll
                    for (int bl = 0; bl < kExB; ++bl)
                        if (bl < nb) v += sb[r][bl] * beta[bl];
                    vw += v * v;
                }
        if (j < K) {
            o[j] = ww;
            o[K + j] = vw;
            o[2 * K + j] = den;
#pragma unroll
            for (int r = 0; r < kExB; ++r)
                if (r < nb) o[(3 + r) * K + j] = s[r];
        }
    }
}

// 2D, one CTA per spectral row a (entries c n0 + a), one grid value per
// thread, with the border rows staged: for an interior row i = a - k,
// wv = sum_r (W0 P V1^T)[i][r]^2 (0 on border rows).
// grid = (n0, items), block = 256; dynamic shared memory 2 (1 + 2k) n1 sizeof(T).
template <typename T>
__global__ void __launch_bounds__(256)
k_ex_rows(const T* __restrict__ spec, const T* __restrict__ D, long long d_psf_stride, int psf_per,
          const T* __restrict__ muT, GcvGeom geo, ExAxis A0, ExAxis A1, int k, T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n0 = A0.n, n1 = A1.n, nb = 2 * k;
    const int a = blockIdx.x;
    const long long item = blockIdx.y;
    const int K = geo.K;
    T* o = out + (item * n0 + a) * (long long)K;
    if (!(a >= k && a < n0 - k)) {
        for (int j = threadIdx.x; j < K; j += blockDim.x) o[j] = 0;
        return;
    }
    T* sa = reinterpret_cast<T*>(smem_raw);     // [1 + nb][n1]
    T* sg = sa + (size_t)(1 + nb) * n1;
    const T* sp = spec + item * geo.S;
    const T* dp = D + (psf_per ? item : 0) * d_psf_stride;
    for (int s = 0; s <= nb; ++s) {
        const int row = s == 0 ? a : A0.bidx[s - 1];
        for (int c = threadIdx.x; c < n1; c += blockDim.x)
            ex_stage<T>(sp, dp, geo, (long long)c * n0 + row, sa[s * n1 + c], sg[s * n1 + c]);
    }
    __syncthreads();
    const T* b0 = reinterpret_cast<const T*>(A0.bhat);
    const T* V1 = reinterpret_cast<const T*>(A1.V);
    const int i = a - k;
    T alpha[kExB];
#pragma unroll
    for (int bk = 0; bk < kExB; ++bk) alpha[bk] = bk < nb ? b0[(size_t)bk * A0.N + i] : (T)0;
    for (int jb = 0; jb < K; jb += blockDim.x) {
        const int j = jb + threadIdx.x;
        const T mu = j < K ? muT[j] : (T)1;
        T u[kExB], ub[kExB][kExB];
#pragma unroll
        for (int r = 0; r < kExB; ++r) {
            u[r] = 0;
#pragma unroll
            for (int bk = 0; bk < kExB; ++bk) ub[r][bk] = 0;
        }
        for (int c = 0; c < n1; ++c) {
            const T P0 = pair_rcp(sa[c] + mu) * sg[c];
            T Pb[kExB];
#pragma unroll
            for (int bk = 0; bk < kExB; ++bk)
                Pb[bk] = bk < nb ? pair_rcp(sa[(1 + bk) * n1 + c] + mu) * sg[(1 + bk) * n1 + c] : (T)0;
#pragma unroll
            for (int r = 0; r < kExB; ++r)
                if (r < nb) {
                    const T v = __ldg(V1 + (size_t)r * n1 + c);
                    u[r] += v * P0;
#pragma unroll
                    for (int bk = 0; bk < kExB; ++bk)
                        if (bk < nb) ub[r][bk] += v * Pb[bk];
                }
        }
        T wv = 0;
#pragma unroll
        for (int r = 0; r < kExB; ++r)
            if (r < nb) {
                T v = u[r];
#pragma unroll
                for (int bk = 0; bk < kExB; ++bk)
                    if (bk < nb) v += alpha[bk] * ub[r][bk];
                wv += v * v;
            }
        if (j < K) o[j] = wv;
    }
}

// 2D: G_ex from the line sums.  Slot s of grid value j (lane) sums, in FP64,
// the columns and rows = s mod kExSlots and its share of
// (V0 P V1^T)[r][r'] = sum_c (V0 P)[r][c] V1[r'][c]; slot 0 adds the slots in
// order.  num = ww + vw + wv + |V0 P V1^T|^2, G = num / den^2.
// grid = (items, ceil(K / 32)), block = (32, kExSlots).
template <typename T>
__global__ void __launch_bounds__(32 * kExSlots)
k_ex_reduce(const T* __restrict__ col_out, const T* __restrict__ row_out, int n0, int n1, int k,
            const double* __restrict__ V1d, int K, double* __restrict__ G) {
    __shared__ double part[4][kExSlots][32];
    __shared__ double vv[kExSlots][kExB * kExB][32];
    const int lane = threadIdx.x, s = threadIdx.y;
    const int j = blockIdx.y * 32 + lane;
    const long long item = blockIdx.x;
    const int nb = 2 * k, nval = 3 + nb;
    double ww = 0, vw = 0, den = 0, wv = 0, m[kExB * kExB];
#pragma unroll
    for (int q = 0; q < kExB * kExB; ++q) m[q] = 0;
    if (j < K) {
        const T* co = col_out + item * (long long)n1 * nval * K;
        for (int c = s; c < n1; c += kExSlots) {
            const T* oc = co + (long long)c * nval * K;
            ww += (double)oc[j];
            vw += (double)oc[K + j];
            den += (double)oc[2 * K + j];
            for (int r = 0; r < nb; ++r) {
                const double sv = (double)oc[(3 + r) * K + j];
                for (int rr = 0; rr < nb; ++rr) m[r * kExB + rr] += sv * V1d[(size_t)rr * n1 + c];
            }
        }
        const T* ro = row_out + item * (long long)n0 * K;
        for (int a = s; a < n0; a += kExSlots) wv += (double)ro[(long long)a * K + j];
    }
    part[0][s][lane] = ww; part[1][s][lane] = vw; part[2][s][lane] = den; part[3][s][lane] = wv;
#pragma unroll
    for (int q = 0; q < kExB * kExB; ++q) vv[s][q][lane] = m[q];
    __syncthreads();
    if (s != 0 || j >= K) return;
    ww = vw = den = wv = 0;
    for (int q = 0; q < kExSlots; ++q) {
        ww += part[0][q][lane]; vw += part[1][q][lane]; den += part[2][q][lane]; wv += part[3][q][lane];
    }
    double vsq = 0;
    for (int q = 0; q < kExB * kExB; ++q) {
        double acc = 0;
        for (int t = 0; t < kExSlots; ++t) acc += vv[t][q][lane];
        vsq += acc * acc;
    }
    G[item * K + j] = (ww + vw + wv + vsq) / (den * den);
}

// 1D: one CTA per problem, one grid value per thread:
// num = sum_i (W P)[i]^2 + sum_r (V P)[r]^2, G = num / (sum sigma)^2.
// grid = items, block = 256; dynamic shared memory 2 n sizeof(T).
template <typename T>
__global__ void __launch_bounds__(256)
k_ex_1d(const T* __restrict__ spec, const T* __restrict__ D, long long d_psf_stride, int psf_per,
        const T* __restrict__ muT, GcvGeom geo, ExAxis A0, int k, double* __restrict__ G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = A0.n, nb = 2 * k;
    T* sa = reinterpret_cast<T*>(smem_raw);
    T* sg = sa + n;
    const long long item = blockIdx.x;
    const T* sp = spec + item * geo.S;
    const T* dp = D + (psf_per ? item : 0) * d_psf_stride;
    for (int a = threadIdx.x; a < n; a += blockDim.x) ex_stage<T>(sp, dp, geo, a, sa[a], sg[a]);
    __syncthreads();
    const T* b0 = reinterpret_cast<const T*>(A0.bhat);
    const T* V0 = reinterpret_cast<const T*>(A0.V);
    const int K = geo.K;
    for (int jb = 0; jb < K; jb += blockDim.x) {
        const int j = jb + threadIdx.x;
        const T mu = j < K ? muT[j] : (T)1;
        T pb[kExB];
#pragma unroll
        for (int b = 0; b < kExB; ++b)
            pb[b] = b < nb ? pair_rcp(sa[A0.bidx[b]] + mu) * sg[A0.bidx[b]] : (T)0;
        T ww = 0, den = 0, s[kExB];
#pragma unroll
        for (int r = 0; r < kExB; ++r) s[r] = 0;
        for (int a = 0; a < n; ++a) {
            const T s0 = pair_rcp(sa[a] + mu);
            const T P0 = s0 * sg[a];
            den += s0;
#pragma unroll
            for (int r = 0; r < kExB; ++r)
                if (r < nb) s[r] += __ldg(V0 + (size_t)r * n + a) * P0;
            if (a >= k && a < n - k) {
                T w = P0;
#pragma unroll
                for (int b = 0; b < kExB; ++b)
                    if (b < nb) w += __ldg(b0 + (size_t)b * A0.N + (a - k)) * pb[b];
                ww += w * w;
            }
        }
        T vsq = 0;
#pragma unroll
        for (int r = 0; r < kExB; ++r)
            if (r < nb) vsq += s[r] * s[r];
        if (j < K) G[item * K + j] = ((double)ww + (double)vsq) / ((double)den * (double)den);
    }
}

// The first minimiser of each problem's curve (NaN never wins).  grid = items, block = 256.
__global__ void k_ex_argmin(const double* __restrict__ G, int K, int* __restrict__ mu_idx) {
    __shared__ double sv[256];
    __shared__ int si[256];
    const long long item = blockIdx.x;
    double best = INFINITY;
    int bi = 0x7fffffff;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        const double v = G[item * K + j];
        const double key = isnan(v) ? INFINITY : v;
        if (key < best || (key == best && j < bi)) { best = key; bi = j; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const double v2 = sv[threadIdx.x + w];
            const int i2 = si[threadIdx.x + w];
            if (v2 < sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) mu_idx[item] = si[0] == 0x7fffffff ? 0 : si[0];
}

void exact_free(hobc_plan_s* p) {
    hobc_exact_s* x = p->exact;
    if (!x) return;
    for (int a = 0; a < 2; ++a) { cudaFree(x->bhat[a]); cudaFree(x->V[a]); cudaFree(x->Vd[a]); }
    cudaFree(x->col_out);
    cudaFree(x->row_out);
    cudaFree(x->G);
    delete x;
    p->exact = nullptr;
}

namespace {

int border_count(int fam) {
    if (fam == HOBC_FAMILY_SINE || fam == HOBC_FAMILY_COSINE) return 1;
    if (fam == HOBC_FAMILY_SINE_CUBIC) return 2;
    if (fam == HOBC_FAMILY_REFLECTIVE || fam == HOBC_FAMILY_PERIODIC) return 0;   // T orthogonal
    return -1;
}

// Builds the row split of each axis and the line-sum buffers on first use.
hobc_status ensure_exact(hobc_plan_s* p) {
    if (p->exact) return HOBC_OK;
    const int k = border_count(p->fam);
    if (k < 0) {
        set_last_error_text("hobc_gcv_exact: real families only (the Fourier family's T_F is complex)");
        return HOBC_ERR_UNSUPPORTED;
    }
    hobc_exact_s* x = new hobc_exact_s();
    p->exact = x;
    x->k = k;
    const bool fp64 = p->prec == HOBC_FP64;
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < p->nax; ++a) {
        const int n = p->ax[a].n;
        x->N[a] = n - 2 * k;
        for (int b = 0; b < 2 * k; ++b) x->bidx[a][b] = b < k ? b : n - 2 * k + b;
        std::vector<double> bhat(1, 0.0), V(1, 0.0);
        if (k > 0) {
            std::vector<double> Tm;
            hobc_status s = axis_matrix(p->fam, n, p->stream, Tm);
            if (s == HOBC_OK) s = split_rows(Tm, n, k, bhat, V);
            if (s != HOBC_OK) { exact_free(p); return s; }
        }
        if (e == cudaSuccess) e = fp64 ? upload<double>(&x->bhat[a], bhat) : upload<float>(&x->bhat[a], bhat);
        if (e == cudaSuccess) e = fp64 ? upload<double>(&x->V[a], V) : upload<float>(&x->V[a], V);
        if (e == cudaSuccess) e = upload<double>((void**)&x->Vd[a], V);
    }
    const size_t B = (size_t)p->desc.batch, K = (size_t)p->K;
    if (p->nax == 2) {
        const size_t n0 = (size_t)p->ax[0].n, n1 = (size_t)p->ax[1].n;
        if (e == cudaSuccess) e = cudaMalloc(&x->col_out, B * n1 * (3 + 2 * k) * K * p->esz);
        if (e == cudaSuccess) e = cudaMalloc(&x->row_out, B * n0 * K * p->esz);
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&x->G, B * K * sizeof(double));
    if (e != cudaSuccess) {
        set_last_error("hobc_gcv_exact (workspace)", e);
        exact_free(p);
        return HOBC_ERR_CUDA;
    }
    return HOBC_OK;
}

ExAxis ex_axis(const hobc_exact_s* x, const hobc_plan_s* p, int a) {
    ExAxis A;
    memset(&A, 0, sizeof(A));
    A.bhat = x->bhat[a];
    A.V = x->V[a];
    A.n = p->ax[a].n;
    A.N = x->N[a];
    for (int b = 0; b < 2 * x->k; ++b) A.bidx[b] = x->bidx[a][b];
    return A;
}

template <typename T>
hobc_status run_gcv_exact(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    hobc_exact_s* x = p->exact;
    GcvGeom geo = exact_geo(p);
    const int B = p->desc.batch, K = p->K, k = x->k;
    const T* sp = reinterpret_cast<const T*>(ghat);
    const T* dp = reinterpret_cast<const T*>(D);
    const T* muT = reinterpret_cast<const T*>(p->muT);
    const long long dps = (long long)p->spec_elems;
    double* Gout = gcv ? gcv : x->G;
    const int threads = std::min(256, (K + 31) / 32 * 32);
    cudaError_t e = cudaSuccess;
    if (p->nax == 1) {
        const int n = p->ax[0].n;
        k_ex_1d<T><<<B, threads, 2 * (size_t)n * sizeof(T), p->stream>>>(sp, dp, dps, p->desc.psf_per_item, muT, geo,
                                                                          ex_axis(x, p, 0), k, Gout);
        p->launches += 1;
    } else {
        const int n0 = p->ax[0].n, n1 = p->ax[1].n;
        const size_t sc = 2 * (size_t)(1 + 2 * k) * n0 * sizeof(T), sr = 2 * (size_t)(1 + 2 * k) * n1 * sizeof(T);
        e = cudaFuncSetAttribute(k_ex_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_ex_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
        if (e != cudaSuccess) { set_last_error("hobc_gcv_exact", e); return HOBC_ERR_CUDA; }
        const ExAxis A0 = ex_axis(x, p, 0), A1 = ex_axis(x, p, 1);
        k_ex_cols<T><<<dim3((unsigned)n1, (unsigned)B), threads, sc, p->stream>>>(
            sp, dp, dps, p->desc.psf_per_item, muT, geo, A0, A1, k, reinterpret_cast<T*>(x->col_out));
        k_ex_rows<T><<<dim3((unsigned)n0, (unsigned)B), threads, sr, p->stream>>>(
            sp, dp, dps, p->desc.psf_per_item, muT, geo, A0, A1, k, reinterpret_cast<T*>(x->row_out));
        k_ex_reduce<T><<<dim3((unsigned)B, (unsigned)((K + 31) / 32)), dim3(32, kExSlots), 0, p->stream>>>(
            reinterpret_cast<const T*>(x->col_out), reinterpret_cast<const T*>(x->row_out), n0, n1, k, x->Vd[1], K,
            Gout);
        p->launches += 3;
    }
    k_ex_argmin<<<B, 256, 0, p->stream>>>(Gout, K, mu_idx);
    p->launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error("hobc_gcv_exact", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

hobc_status gcv_exact_dispatch(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    return p->prec == HOBC_FP64 ? run_gcv_exact<double>(p, ghat, D, gcv, mu_idx)
                                : run_gcv_exact<float>(p, ghat, D, gcv, mu_idx);
}

}  // namespace
}  // namespace hobc

using namespace hobc;

extern "C" {

hobc_status hobc_gcv_exact(hobc_plan* p, const void* ghat_dev, const void* d_dev, double* gcv_dev, int* mu_index_dev) {
    if (!p || !ghat_dev || !d_dev || !mu_index_dev) return HOBC_ERR_ARG;
    hobc_status s = ensure_exact(p);
    if (s != HOBC_OK) return s;
    p->launches = 0;
    return gcv_exact_dispatch(p, ghat_dev, d_dev, gcv_dev, mu_index_dev);
}

hobc_status hobc_deblur_exact(hobc_plan* p, const void* g_dev, const void* psf_dev, void* f_dev, int* mu_index_dev,
                              double* gcv_dev) {
    if (!p || !g_dev || !psf_dev || !f_dev) return HOBC_ERR_ARG;
    if (g_dev == f_dev) return HOBC_ERR_ARG;
    hobc_status s = ensure_exact(p);
    if (s != HOBC_OK) return s;
    p->launches = 0;
    int* mi = mu_index_dev ? mu_index_dev : p->mu_idx;
    const bool fp64 = p->prec == HOBC_FP64;
    s = fp64 ? run_eig<double>(p, psf_dev, p->D) : run_eig<float>(p, psf_dev, p->D);
    if (s == HOBC_OK) s = fp64 ? run_analysis<double>(p, g_dev, p->G) : run_analysis<float>(p, g_dev, p->G);
    if (s == HOBC_OK) s = gcv_exact_dispatch(p, p->G, p->D, gcv_dev, mi);
    if (s == HOBC_OK)
        s = fp64 ? run_filter_synthesis<double>(p, p->G, p->D, mi, f_dev)
                 : run_filter_synthesis<float>(p, p->G, p->D, mi, f_dev);
    return s;
}

}  // extern "C"
