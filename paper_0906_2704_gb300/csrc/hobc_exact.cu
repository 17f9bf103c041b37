// The exact GCV functional of Eq. (eq:gcv) (include/hobc_exact.h).  Per plan,
// once: T_a of each axis from the FP64 synthesis path, split by rows on the
// host (FP64): the interior rows are X_a^H W_a with X_a^H unitary and
// W_a = [bhat_L | I | bhat_R], the 2k extension rows (at the border indices)
// are V_a.  Then
//   ||T_0 P T_1^T||^2 = ||W0 P W1^T||^2 + ||V0 P W1^T||^2 + ||W0 P V1^T||^2
//                       + ||V0 P V1^T||^2,
// every term a sum of squares (no cancellation between large terms, which
// the Gram form |P|^2 + P^H (T^H T - I) P suffers: T_C at n = 1024 has
// condition ~2e4).  Per call: one CTA per stored spectral column, one per
// spectral row, an FP64 reduction and the argmin; 1D plans one CTA per
// problem.  The Fourier family stores half of the last axis: a full column of
// the other half is the conjugate of a stored column with its rows mapped
// t -> -t, so column sums carry the pair weight 2, and row sums and
// V0 P V1^T add the partner entries explicitly.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/hobc_exact.h"
#include "hobc_internal.h"
#include "hobc_kernels.cuh"

typedef std::complex<double> cdx;

struct hobc_exact_s {
    int k;                 // border vectors per side (1: degrees 1 and 2, 2: degree 3, 0: orthogonal T)
    int cplx;              // Fourier family: complex T and a half spectrum on the last axis
    int N[2];              // interior length n_a - 2k
    int bidx[2][4];        // border indices of each axis: 0..k-1, n-k..n-1
    void* bhat[2];         // [2k][N_a] plan precision (complex for the Fourier family)
    void* V[2];            // [2k][n_a] plan precision: the extension rows of T_a
    void* Vd[2];           // [2k][n_a] FP64 copy of V_a (the V_0 P V_1^T term)
    void* col_out;         // [batch][stored columns][2 + 2k (x2 complex)][K]: ww, den, (V0 P)[r][c]
    void* row_out;         // [batch][n_0][2k (x2 complex)][K]: (P V1^T)[a][r]
    double* G;             // [batch][K] when the caller passes no curve
    // coarse-to-fine search (allocated on its first call)
    int* s_idx;            // [batch][32] grid indices of a level
    void* s_mu;            // [batch][32] their mu, plan precision
    double* s_G;           // [batch][32] G_ex at them
    double* s_best;        // [batch] G_ex of the incumbent
    double* red;           // reduction partials [batch][P][K][4 + 2 NB^2]
    size_t red_cap;        // doubles allocated in red
};

namespace hobc {

constexpr int kExKMax = 2;             // border vectors per side at most (degree 3)
constexpr int kExB = 2 * kExKMax;
constexpr int kExSlots = 4;            // reduction: line slices per grid value
constexpr int kExCB = 4;               // stored columns per CTA of the column pass
constexpr int kExParts = 16;           // reduction: line partitions (CTAs per grid value block) at most

// ------------------------------------------------- real or complex entries
__device__ __forceinline__ float xm(float a, float b) { return a * b; }
__device__ __forceinline__ double xm(double a, double b) { return a * b; }
__device__ __forceinline__ float2 xm(float2 a, float2 b) { return cmul<float>(a, b); }
__device__ __forceinline__ double2 xm(double2 a, double2 b) { return cmul<double>(a, b); }
__device__ __forceinline__ float xa(float a, float b) { return a + b; }
__device__ __forceinline__ double xa(double a, double b) { return a + b; }
__device__ __forceinline__ float2 xa(float2 a, float2 b) { return cadd<float>(a, b); }
__device__ __forceinline__ double2 xa(double2 a, double2 b) { return cadd<double>(a, b); }
__device__ __forceinline__ float xc(float a) { return a; }
__device__ __forceinline__ double xc(double a) { return a; }
__device__ __forceinline__ float2 xc(float2 a) { return cconj<float>(a); }
__device__ __forceinline__ double2 xc(double2 a) { return cconj<double>(a); }
__device__ __forceinline__ float xs(float a, float s) { return a * s; }
__device__ __forceinline__ double xs(double a, double s) { return a * s; }
__device__ __forceinline__ float2 xs(float2 a, float s) { return cscale<float>(a, s); }
__device__ __forceinline__ double2 xs(double2 a, double s) { return cscale<double>(a, s); }
template <typename E> __device__ __forceinline__ E xz();
template <> __device__ __forceinline__ float xz<float>() { return 0.f; }
template <> __device__ __forceinline__ double xz<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 xz<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 xz<double2>() { return make_double2(0.0, 0.0); }

// Butterfly sums over the rs adjacent lanes that share a grid value (rs a power
// of two <= 32; every lane of the warp takes part).
__device__ __forceinline__ float shx(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shx(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float2 shx(float2 v, int o) { return make_float2(shx(v.x, o), shx(v.y, o)); }
__device__ __forceinline__ double2 shx(double2 v, int o) { return make_double2(shx(v.x, o), shx(v.y, o)); }
template <typename E> __device__ __forceinline__ E lane_sum(E v, int rs) {
    for (int o = rs / 2; o > 0; o >>= 1) v = xa(v, shx(v, o));
    return v;
}

// Fourier half spectrum along an axis of n (N = n - 2): spectral index of a
// stored entry, whether it stands alone (no conjugate partner), and t -> -t.
__device__ __forceinline__ int hx_t(int c, int n, int W) { return c == W - 1 ? n - 1 : c; }
__device__ __forceinline__ bool hx_self(int c, int n, int W) { return c == 0 || c == W - 1 || c == 1 || 2 * (c - 1) == n - 2; }
__device__ __forceinline__ int hx_neg(int t, int n) {
    const int N = n - 2;
    return (t == 0 || t == n - 1) ? t : 1 + (N - (t - 1)) % N;
}

namespace {

// Column t of T_X of one axis (T[i * n + t]) from the FP64 synthesis path.
// Real families: synthesis of e_t.  Fourier family (real signals from half
// spectra): a unit at stored bin c gives T[:, t] + T[:, -t] = 2 Re T[:, t] and
// an imaginary unit gives -2 Im T[:, t]; borders and self-conjugate bins are
// real columns; T[:, -t] = conj T[:, t].
hobc_status axis_matrix(int fam, int n, cudaStream_t st, std::vector<cdx>& T) {
    const bool F = fam == HOBC_FAMILY_FOURIER;
    const int N = n - 2;
    const int W = F ? N / 2 + 3 : n;
    const int items = F ? 2 * W : n;
    hobc_plan_desc q;
    memset(&q, 0, sizeof(q));
    q.ndim = 1; q.n[0] = n; q.psf[0] = 1; q.family = (hobc_family)fam; q.psf_symmetric = 1;
    q.bc_degree = fam == HOBC_FAMILY_SINE ? 1 : fam == HOBC_FAMILY_SINE_CUBIC ? 3 : fam == HOBC_FAMILY_COSINE_QUARTIC ? 4 : 2;
    q.L = HOBC_L_IDENTITY; q.prec = HOBC_FP64; q.n_mu = 1; q.batch = items; q.psf_per_item = 0;
    const double one = 1.0;
    hobc_plan* ip = nullptr;
    hobc_status s = hobc_plan_create(&q, &one, st, &ip);
    if (s != HOBC_OK) return s;
    const size_t in_per = F ? 2 * (size_t)W : (size_t)n;        // doubles per input item
    std::vector<double> in((size_t)items * in_per, 0.0), Y((size_t)items * n);
    if (F)
        for (int c = 0; c < W; ++c) {
            in[(size_t)(2 * c) * in_per + 2 * c] = 1.0;          // real unit at stored c
            in[(size_t)(2 * c + 1) * in_per + 2 * c + 1] = 1.0;  // imaginary unit at stored c
        }
    else
        for (int t = 0; t < n; ++t) in[(size_t)t * in_per + t] = 1.0;
    double *I = nullptr, *out = nullptr;
    cudaError_t e = cudaMalloc((void**)&I, in.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&out, Y.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(I, in.data(), in.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) s = hobc_synthesis(ip, I, out);
    if (e == cudaSuccess && s == HOBC_OK) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && s == HOBC_OK) e = cudaMemcpy(Y.data(), out, Y.size() * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(I);
    cudaFree(out);
    hobc_plan_destroy(ip);
    if (s != HOBC_OK) return s;
    if (e != cudaSuccess) { set_last_error("hobc_gcv_exact (transform matrix)", e); return HOBC_ERR_CUDA; }
    T.assign((size_t)n * n, cdx(0, 0));
    if (!F) {
        for (int t = 0; t < n; ++t)
            for (int i = 0; i < n; ++i) T[(size_t)i * n + t] = Y[(size_t)t * n + i];
        return HOBC_OK;
    }
    for (int c = 0; c < W; ++c) {
        const int t = c == W - 1 ? n - 1 : c;
        const bool self = c == 0 || c == W - 1 || c == 1 || 2 * (c - 1) == N;
        const double* yr = &Y[(size_t)(2 * c) * n];
        const double* yi = &Y[(size_t)(2 * c + 1) * n];
        if (self) {
            for (int i = 0; i < n; ++i) T[(size_t)i * n + t] = yr[i];
        } else {
            const int tn = 1 + (N - (t - 1)) % N;
            for (int i = 0; i < n; ++i) {
                const cdx v(0.5 * yr[i], -0.5 * yi[i]);
                T[(size_t)i * n + t] = v;
                T[(size_t)i * n + tn] = std::conj(v);
            }
        }
    }
    return HOBC_OK;
}

// The row split of T (k border indices per side): interior rows k..n-k-1 are
// X^H [bhat_L | I | bhat_R] with X^H = T[interior][interior] unitary, and the
// extension rows (the border indices) are V.  Checks the unitarity.
hobc_status split_rows(const std::vector<cdx>& T, int n, int k, std::vector<cdx>& bhat, std::vector<cdx>& V) {
    const int N = n - 2 * k;
    double dev = 0;
    for (int i = 0; i < N; ++i)                 // rows of X^H are orthonormal
        for (int j = i; j < N; ++j) {
            cdx acc(0, 0);
            for (int m = 0; m < N; ++m) acc += T[(size_t)(k + i) * n + k + m] * std::conj(T[(size_t)(k + j) * n + k + m]);
            dev = std::max(dev, std::abs(acc - cdx(i == j ? 1.0 : 0.0, 0.0)));
        }
    if (dev > 1e-10) {
        set_last_error_text("hobc_gcv_exact: the interior block of T is not unitary");
        return HOBC_ERR_UNSUPPORTED;
    }
    bhat.assign((size_t)std::max(2 * k * N, 1), cdx(0, 0));
    V.assign((size_t)std::max(2 * k * n, 1), cdx(0, 0));
    for (int b = 0; b < 2 * k; ++b) {
        const int col = b < k ? b : n - 2 * k + b;
        for (int i = 0; i < N; ++i) {           // (X t_int)[i] = sum_m conj(X^H[m][i]) T[k + m][col]
            cdx acc(0, 0);
            for (int m = 0; m < N; ++m) acc += std::conj(T[(size_t)(k + m) * n + k + i]) * T[(size_t)(k + m) * n + col];
            bhat[(size_t)b * N + i] = acc;
        }
        for (int a = 0; a < n; ++a) V[(size_t)b * n + a] = T[(size_t)col * n + a];
    }
    return HOBC_OK;
}

// Device copy in the plan's precision: real parts only, or (re, im) pairs.
template <typename T> cudaError_t upload(void** dst, const std::vector<cdx>& v, bool cplx) {
    std::vector<T> w(v.size() * (cplx ? 2 : 1));
    for (size_t i = 0; i < v.size(); ++i) {
        if (cplx) { w[2 * i] = (T)v[i].real(); w[2 * i + 1] = (T)v[i].imag(); }
        else w[i] = (T)v[i].real();
    }
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
    int n, N, W;           // W: stored entries along the axis (half spectrum on the Fourier family's last axis)
    int bidx[kExB];        // border spectral indices
    int bcol[kExB];        // their stored positions
};

}  // namespace

// a and ghat of stored entry e: entries with s = 0 carry a = inf (sigma = 0,
// so they drop out as in the approximation).
template <typename T, bool CPLX>
__device__ __forceinline__ void ex_stage(const typename ElemT<T, CPLX>::t* sp, const typename ElemT<T, CPLX>::t* dp,
                                         const GcvGeom& geo, long long e, T& a, typename ElemT<T, CPLX>::t& g) {
    typedef typename ElemT<T, CPLX>::t E;
    const typename Pack4<T>::t v = gcv_term<T, CPLX>(sp[e], dp[e], geo, e);
    const bool live = v.z > (T)0;
    a = live ? v.x : (T)INFINITY;
    g = live ? sp[e] : xz<E>();
}

// 2D, one CTA per kExCB consecutive stored spectral columns (entries
// c n0 + a), one grid value per thread, with the border columns staged once
// for all of them.  Per column (spectral index t): for an interior column
// (j = t - k), ww = sum_i |(W0 P W1^T)[i][j]|^2; for every column, den =
// sum sigma and the projections (V0 P)[r][c].  ww and den carry the column's
// pair weight (2 for a stored Fourier column that stands for a conjugate
// pair).  The V0 P W1^T term is formed from the projections in k_ex_reduce.
// grid = (ceil(stored columns / kExCB), items), block <= 256;
// dynamic shared memory (kExCB + 2k) n0 (sizeof(T) + sizeof(E)).
template <typename T, bool CPLX, int NB, bool SL>
__global__ void __launch_bounds__(256)
k_ex_cols(const typename ElemT<T, CPLX>::t* __restrict__ spec, const typename ElemT<T, CPLX>::t* __restrict__ D,
          long long d_psf_stride, int psf_per, const T* __restrict__ muT, int mu_stride, int rs_arg, GcvGeom geo,
          ExAxis A0, ExAxis A1, T* __restrict__ out) {
    typedef typename ElemT<T, CPLX>::t E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int nb = NB, k = NB / 2, NB1 = NB > 0 ? NB : 1, ns = kExCB + NB;
    __shared__ E sbeta[kExCB][NB1];
    const int n0 = A0.n, n1 = A1.n, W1 = A1.W;
    E* sg = reinterpret_cast<E*>(smem_raw);                      // [ns][n0]
    T* sa = reinterpret_cast<T*>(sg + (size_t)ns * n0);          // [ns][n0]
    const int c0 = blockIdx.x * kExCB;
    const long long item = blockIdx.y;
    const E* sp = spec + item * geo.S;
    const E* dp = D + (psf_per ? item : 0) * d_psf_stride;
    for (int s = 0; s < ns; ++s) {
        const int col = s < kExCB ? min(c0 + s, W1 - 1) : A1.bcol[s - kExCB];
        for (int a = threadIdx.x; a < n0; a += blockDim.x)
            ex_stage<T, CPLX>(sp, dp, geo, (long long)col * n0 + a, sa[s * n0 + a], sg[s * n0 + a]);
    }
    const E* b1 = reinterpret_cast<const E*>(A1.bhat);
    if (threadIdx.x < kExCB * NB1) {
        const int q = threadIdx.x / NB1, bl = threadIdx.x % NB1;
        const int t = CPLX ? hx_t(min(c0 + q, W1 - 1), n1, W1) : min(c0 + q, W1 - 1);
        sbeta[q][bl] = (bl < nb && t >= k && t < n1 - k) ? b1[(size_t)bl * A1.N + (t - k)] : xz<E>();
    }
    __syncthreads();
    const E* b0 = reinterpret_cast<const E*>(A0.bhat);
    const E* V0 = reinterpret_cast<const E*>(A0.V);
    int tq[kExCB];
    bool inter[kExCB];
#pragma unroll
    for (int q = 0; q < kExCB; ++q) {
        const int cq = min(c0 + q, W1 - 1);
        tq[q] = CPLX ? hx_t(cq, n1, W1) : cq;
        inter[q] = c0 + q < W1 && tq[q] >= k && tq[q] < n1 - k;
    }
    const int K = geo.K;
    const int nval = 2 + nb * (CPLX ? 2 : 1);
    const int rs = SL ? rs_arg : 1;           // lanes per grid value (1: one value per thread)
    const int sl = threadIdx.x % rs, jpb = blockDim.x / rs;
    const T* mup = muT + item * mu_stride;
    for (int jb = 0; jb < K; jb += jpb) {
        const int j = jb + threadIdx.x / rs;
        const T mu = j < K ? mup[j] : (T)1;
        E gam[kExCB][NB1];                    // P[bk][t] + sum_bl P[bk][bl] bhat1[bl][j(t)]
#pragma unroll
        for (int bk = 0; bk < NB; ++bk) {
            E corner[NB1];
            const int ar = bk < nb ? A0.bidx[bk] : 0;
#pragma unroll
            for (int bl = 0; bl < NB; ++bl)
                corner[bl] = (bk < nb && bl < nb)
                                 ? xs(sg[(kExCB + bl) * n0 + ar], pair_rcp(sa[(kExCB + bl) * n0 + ar] + mu)) : xz<E>();
#pragma unroll
            for (int q = 0; q < kExCB; ++q) {
                E gv = xz<E>();
                if (bk < nb) {
                    gv = xs(sg[q * n0 + ar], pair_rcp(sa[q * n0 + ar] + mu));
#pragma unroll
                    for (int bl = 0; bl < NB; ++bl)
                        if (bl < nb) gv = xa(gv, xm(corner[bl], sbeta[q][bl]));
                }
                gam[q][bk] = gv;
            }
        }
        T ww[kExCB], den[kExCB];
        E s[kExCB][NB1];
#pragma unroll
        for (int q = 0; q < kExCB; ++q) {
            ww[q] = 0;
            den[q] = 0;
#pragma unroll
            for (int r = 0; r < NB; ++r) s[q][r] = xz<E>();
        }
        for (int a = sl; a < n0; a += rs) {
            E Pb[NB1], v0[NB1], bb[NB1];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                Pb[b] = b < nb ? xs(sg[(kExCB + b) * n0 + a], pair_rcp(sa[(kExCB + b) * n0 + a] + mu)) : xz<E>();
                v0[b] = b < nb ? V0[(size_t)b * n0 + a] : xz<E>();
            }
            const bool ai = a >= k && a < n0 - k;
#pragma unroll
            for (int b = 0; b < NB; ++b) bb[b] = (ai && b < nb) ? b0[(size_t)b * A0.N + (a - k)] : xz<E>();
#pragma unroll
            for (int q = 0; q < kExCB; ++q) {
                const T s0 = pair_rcp(sa[q * n0 + a] + mu);
                const E P0 = xs(sg[q * n0 + a], s0);
                den[q] += s0;
#pragma unroll
                for (int r = 0; r < NB; ++r)
                    if (r < nb) s[q][r] = xa(s[q][r], xm(v0[r], P0));
                if (inter[q] && ai) {
                    E w = P0;
#pragma unroll
                    for (int b = 0; b < NB; ++b)
                        if (b < nb) w = xa(xa(w, xm(Pb[b], sbeta[q][b])), xm(bb[b], gam[q][b]));
                    ww[q] += abs2_of(w);
                }
            }
        }
        if (rs > 1)
#pragma unroll
            for (int q = 0; q < kExCB; ++q) {
                ww[q] = lane_sum(ww[q], rs);
                den[q] = lane_sum(den[q], rs);
#pragma unroll
                for (int r = 0; r < NB; ++r) s[q][r] = lane_sum(s[q][r], rs);
            }
        if (j < K && sl == 0)
#pragma unroll
            for (int q = 0; q < kExCB; ++q) {
                const int c = c0 + q;
                if (c >= W1) continue;
                const T wgt = (CPLX && !hx_self(c, n1, W1)) ? (T)2 : (T)1;
                T* o = out + (item * W1 + c) * (long long)nval * K;
                o[j] = wgt * ww[q];
                o[K + j] = wgt * den[q];
#pragma unroll
                for (int r = 0; r < NB; ++r)
                    if (r < nb) {
                        if constexpr (CPLX) {
                            o[(2 + 2 * r) * K + j] = s[q][r].x;
                            o[(3 + 2 * r) * K + j] = s[q][r].y;
                        } else {
                            o[(2 + r) * K + j] = s[q][r];
                        }
                    }
            }
    }
}

// 2D, the projections u_r = (P V1^T)[a][r] of every spectral row a over the
// full row, one grid value per thread.  Real families: one CTA per row.
// Fourier family: one CTA per row pair (a, -a) (a row that is its own
// partner alone), grid.x = the W0 = N0/2 + 3 representatives a of the pairs;
// a stored column c that stands for a conjugate pair adds the partner entry
// P[a][-t] = conj(P[-a][t]) at V1's column -t, so the two staged rows give
// both rows' sums from one reciprocal per stored entry.  The W0 P V1^T term
// is formed from the projections in k_ex_reduce.
// dynamic shared memory (1 or 2) W1 (sizeof(T) + sizeof(E)).
template <typename T, bool CPLX, int NB, bool SL>
__global__ void __launch_bounds__(256)
k_ex_rows(const typename ElemT<T, CPLX>::t* __restrict__ spec, const typename ElemT<T, CPLX>::t* __restrict__ D,
          long long d_psf_stride, int psf_per, const T* __restrict__ muT, int mu_stride, int rs_arg, GcvGeom geo,
          ExAxis A0, ExAxis A1, T* __restrict__ out) {
    typedef typename ElemT<T, CPLX>::t E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int nb = NB, NB1 = NB > 0 ? NB : 1;
    const int n0 = A0.n, n1 = A1.n, W1 = A1.W;
    const int a = CPLX ? hx_t(blockIdx.x, n0, (n0 - 2) / 2 + 3) : (int)blockIdx.x;
    const int ap = CPLX ? hx_neg(a, n0) : a;                      // partner row
    const bool two = ap != a;
    const long long item = blockIdx.y;
    const int K = geo.K;
    const int nval = nb * (CPLX ? 2 : 1);
    const int ns = CPLX ? 2 : 1;
    E* sg = reinterpret_cast<E*>(smem_raw);                      // [ns][W1]
    T* sa = reinterpret_cast<T*>(sg + (size_t)ns * W1);          // [ns][W1]
    const E* sp = spec + item * geo.S;
    const E* dp = D + (psf_per ? item : 0) * d_psf_stride;
    for (int s = 0; s < ns; ++s) {
        const int row = s == 0 ? a : ap;
        for (int c = threadIdx.x; c < W1; c += blockDim.x)
            ex_stage<T, CPLX>(sp, dp, geo, (long long)c * n0 + row, sa[s * W1 + c], sg[s * W1 + c]);
    }
    __syncthreads();
    const E* V1 = reinterpret_cast<const E*>(A1.V);
    T* o = out + (item * n0 + a) * (long long)nval * K;
    T* op = out + (item * n0 + ap) * (long long)nval * K;
    const int rs = SL ? rs_arg : 1;           // lanes per grid value (1: one value per thread)
    const int sl = threadIdx.x % rs, jpb = blockDim.x / rs;
    const T* mup = muT + item * mu_stride;
    for (int jb = 0; jb < K; jb += jpb) {
        const int j = jb + threadIdx.x / rs;
        const T mu = j < K ? mup[j] : (T)1;
        E u[NB1], up[NB1];
#pragma unroll
        for (int r = 0; r < NB1; ++r) { u[r] = xz<E>(); up[r] = xz<E>(); }
        for (int c = sl; c < W1; c += rs) {
            const int t = CPLX ? hx_t(c, n1, W1) : c;
            const E P0 = xs(sg[c], pair_rcp(sa[c] + mu));
            if constexpr (CPLX) {
                const E Pq = two ? xs(sg[W1 + c], pair_rcp(sa[W1 + c] + mu)) : P0;   // row -a
                const bool pair = !hx_self(c, n1, W1);
                const int tn = hx_neg(t, n1);
#pragma unroll
                for (int r = 0; r < NB; ++r) {
                    const E v = V1[(size_t)r * n1 + t];
                    u[r] = xa(u[r], xm(v, P0));
                    up[r] = xa(up[r], xm(v, Pq));
                    if (pair) {
                        const E vn = V1[(size_t)r * n1 + tn];
                        u[r] = xa(u[r], xm(vn, xc(Pq)));
                        up[r] = xa(up[r], xm(vn, xc(P0)));
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < NB; ++r) u[r] = xa(u[r], xm(V1[(size_t)r * n1 + t], P0));
            }
        }
        if (rs > 1)
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                u[r] = lane_sum(u[r], rs);
                if constexpr (CPLX) up[r] = lane_sum(up[r], rs);
            }
        if (j < K && sl == 0)
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                if constexpr (CPLX) {
                    o[(2 * r) * K + j] = u[r].x;
                    o[(2 * r + 1) * K + j] = u[r].y;
                    if (two) {
                        op[(2 * r) * K + j] = up[r].x;
                        op[(2 * r + 1) * K + j] = up[r].y;
                    }
                } else {
                    o[r * K + j] = u[r];
                }
            }
    }
}

// 2D: G_ex from the line sums, in two kernels.  k_ex_reduce: CTA (item,
// y, z) takes grid values y*jpc .. y*jpc + jpc - 1, jpc = 32 / LS (LS = 2^ls_log2
// adjacent lanes per value), and the stored columns and rows c = (z kExSlots +
// s) LS + l mod (P kExSlots LS) for slot s, lane offset l and P = gridDim.z:
// the column sums ww and den, the column terms |(V0 P W1^T)[r][j]|^2 =
// |(V0 P)[r][c] + sum_bl (V0 P)[r][bl] bhat1[bl][j]|^2 (pair-weighted), the
// row terms |(W0 P V1^T)[i][r]|^2 = |u_r(a) + sum_bk bhat0[bk][i] u_r(bk)|^2,
// and its share of (V0 P V1^T)[r][r'] = sum over full columns of (V0 P)[r][t]
// V1[r'][t] (a stored Fourier column that stands for a pair adds
// conj((V0 P)[r][c]) at V1's column -t).  Line terms in the working precision,
// sums in FP64; the lanes of a value and the slots are added in a fixed order
// and the CTA's sums go to part[item][z][j][0 .. 4 + 2 NB^2).  k_ex_finish adds
// the P partitions in order and forms num = ww + vw + wv + |V0 P V1^T|^2,
// G = num / den^2.  grid = (items, ceil(K / jpc), P), block = (32, kExSlots).
template <typename T, bool CPLX, int NB>
__global__ void __launch_bounds__(32 * kExSlots)
k_ex_reduce(const T* __restrict__ col_out, const T* __restrict__ row_out, ExAxis A0, ExAxis A1,
            const double* __restrict__ V1d, int K, int ls_log2, double* __restrict__ part_out) {
    typedef typename ElemT<T, CPLX>::t E;
    constexpr int nb = NB, k = NB / 2, NB1 = NB > 0 ? NB : 1, NV = 4 + 2 * NB1 * NB1;
    __shared__ double part[NV][kExSlots][32];
    const int LS = 1 << ls_log2;
    const int lane = threadIdx.x, s = threadIdx.y;
    const int jl = lane >> ls_log2, l = lane & (LS - 1), jpc = 32 >> ls_log2;
    const int j = blockIdx.y * jpc + jl;
    const long long item = blockIdx.x;
    const int z = blockIdx.z, P = gridDim.z;
    const int stride = P * kExSlots * LS, start = (z * kExSlots + s) * LS + l;
    const int n0 = A0.n, n1 = A1.n, W1 = A1.W;
    const int cv = nb * (CPLX ? 2 : 1), ncol = 2 + cv;
    const E* b0 = reinterpret_cast<const E*>(A0.bhat);
    const E* b1 = reinterpret_cast<const E*>(A1.bhat);
    double ww = 0, vw = 0, den = 0, wv = 0, mr[NB1 * NB1], mi[NB1 * NB1];
#pragma unroll
    for (int q = 0; q < NB1 * NB1; ++q) { mr[q] = 0; mi[q] = 0; }
    auto ld = [&](const T* base, int idx) -> E {          // projection idx of a line's output
        if constexpr (CPLX) { E v; v.x = base[(2 * idx) * K + j]; v.y = base[(2 * idx + 1) * K + j]; return v; }
        else return base[idx * K + j];
    };
    if (j < K) {
        const T* co = col_out + item * (long long)W1 * ncol * K;
        const T* ro = row_out + item * (long long)n0 * cv * K;
        E sB[NB1][NB1], uB[NB1][NB1];      // projections of the border columns / rows
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                sB[b][r] = (b < nb && r < nb) ? ld(co + (long long)A1.bcol[b] * ncol * K + 2 * K, r) : xz<E>();
                uB[b][r] = (b < nb && r < nb) ? ld(ro + (long long)A0.bidx[b] * cv * K, r) : xz<E>();
            }
        for (int c = start; c < W1; c += stride) {
            const T* oc = co + (long long)c * ncol * K;
            ww += (double)oc[j];
            den += (double)oc[K + j];
            const int t = CPLX ? hx_t(c, n1, W1) : c;
            const bool pair = CPLX && !hx_self(c, n1, W1);
            const bool inter = t >= k && t < n1 - k;
            T term = 0;
            for (int r = 0; r < nb; ++r) {
                const E sr = ld(oc + 2 * K, r);
                if (inter) {
                    E v = sr;
                    for (int b = 0; b < nb; ++b) v = xa(v, xm(sB[b][r], b1[(size_t)b * A1.N + (t - k)]));
                    term += abs2_of(v);
                }
                double sre, sim;
                if constexpr (CPLX) { sre = sr.x; sim = sr.y; } else { sre = sr; sim = 0.0; }
                for (int rr = 0; rr < nb; ++rr) {
                    const double vr = CPLX ? V1d[2 * ((size_t)rr * n1 + t)] : V1d[(size_t)rr * n1 + t];
                    const double vi = CPLX ? V1d[2 * ((size_t)rr * n1 + t) + 1] : 0.0;
                    mr[r * NB1 + rr] += sre * vr - sim * vi;
                    mi[r * NB1 + rr] += sre * vi + sim * vr;
                    if (pair) {                 // conj(s) at column -t
                        const int tn = hx_neg(t, n1);
                        const double pr = V1d[2 * ((size_t)rr * n1 + tn)], pim = V1d[2 * ((size_t)rr * n1 + tn) + 1];
                        mr[r * NB1 + rr] += sre * pr + sim * pim;
                        mi[r * NB1 + rr] += sre * pim - sim * pr;
                    }
                }
            }
            vw += (pair ? 2.0 : 1.0) * (double)term;
        }
        for (int a = start; a < n0; a += stride) {
            if (a < k || a >= n0 - k) continue;
            const T* orow = ro + (long long)a * cv * K;
            T term = 0;
            for (int r = 0; r < nb; ++r) {
                E v = ld(orow, r);
                for (int b = 0; b < nb; ++b) v = xa(v, xm(b0[(size_t)b * A0.N + (a - k)], uB[b][r]));
                term += abs2_of(v);
            }
            wv += (double)term;
        }
    }
    for (int o = LS / 2; o > 0; o >>= 1) {           // the lanes of one grid value
        ww += shx(ww, o); vw += shx(vw, o); den += shx(den, o); wv += shx(wv, o);
#pragma unroll
        for (int q = 0; q < NB1 * NB1; ++q) { mr[q] += shx(mr[q], o); mi[q] += shx(mi[q], o); }
    }
    if (l == 0) {
        part[0][s][jl] = ww; part[1][s][jl] = vw; part[2][s][jl] = den; part[3][s][jl] = wv;
#pragma unroll
        for (int q = 0; q < NB1 * NB1; ++q) { part[4 + 2 * q][s][jl] = mr[q]; part[5 + 2 * q][s][jl] = mi[q]; }
    }
    __syncthreads();
    if (s != 0 || l != 0 || j >= K) return;
    double* o = part_out + ((item * P + z) * (long long)K + j) * NV;
    for (int v = 0; v < NV; ++v) {
        double acc = 0;
        for (int q = 0; q < kExSlots; ++q) acc += part[v][q][jl];
        o[v] = acc;
    }
}

// G_ex of every (item, grid value) from the P partitions of k_ex_reduce, added
// in partition order.  grid = items, block = min(256, K rounded up to 32).
template <int NB>
__global__ void k_ex_finish(const double* __restrict__ part_in, int K, int P, double* __restrict__ G) {
    constexpr int NB1 = NB > 0 ? NB : 1, NV = 4 + 2 * NB1 * NB1;
    const long long item = blockIdx.x;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        double acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = 0;
        for (int z = 0; z < P; ++z) {
            const double* pz = part_in + ((item * P + z) * (long long)K + j) * NV;
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += pz[v];
        }
        double vsq = 0;
#pragma unroll
        for (int q = 0; q < NB1 * NB1; ++q) vsq += acc[4 + 2 * q] * acc[4 + 2 * q] + acc[5 + 2 * q] * acc[5 + 2 * q];
        G[item * K + j] = (acc[0] + acc[1] + acc[3] + vsq) / (acc[2] * acc[2]);
    }
}

// 1D: one CTA per problem, one grid value per thread:
// num = sum_i |(W P)[i]|^2 + sum_r |(V P)[r]|^2, G = num / (sum sigma)^2 (Fourier
// half spectrum: pair weights on the first two sums, partner entries in V P).
// grid = items, block <= 256; dynamic shared memory W (sizeof(T) + sizeof(E)).
template <typename T, bool CPLX, int NB, bool SL>
__global__ void __launch_bounds__(256)
k_ex_1d(const typename ElemT<T, CPLX>::t* __restrict__ spec, const typename ElemT<T, CPLX>::t* __restrict__ D,
        long long d_psf_stride, int psf_per, const T* __restrict__ muT, int mu_stride, int rs_arg, GcvGeom geo,
        ExAxis A0, double* __restrict__ G) {
    typedef typename ElemT<T, CPLX>::t E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int nb = NB, k = NB / 2, NB1 = NB > 0 ? NB : 1;
    const int n = A0.n, W = A0.W;
    E* sg = reinterpret_cast<E*>(smem_raw);
    T* sa = reinterpret_cast<T*>(sg + W);
    const long long item = blockIdx.x;
    const E* sp = spec + item * geo.S;
    const E* dp = D + (psf_per ? item : 0) * d_psf_stride;
    for (int c = threadIdx.x; c < W; c += blockDim.x) ex_stage<T, CPLX>(sp, dp, geo, c, sa[c], sg[c]);
    __syncthreads();
    const E* b0 = reinterpret_cast<const E*>(A0.bhat);
    const E* V0 = reinterpret_cast<const E*>(A0.V);
    const int K = geo.K;
    const int rs = SL ? rs_arg : 1;           // lanes per grid value (1: one value per thread)
    const int sl = threadIdx.x % rs, jpb = blockDim.x / rs;
    const T* mup = muT + item * mu_stride;
    for (int jb = 0; jb < K; jb += jpb) {
        const int j = jb + threadIdx.x / rs;
        const T mu = j < K ? mup[j] : (T)1;
        E pb[NB1];
#pragma unroll
        for (int b = 0; b < NB; ++b)
            pb[b] = b < nb ? xs(sg[A0.bcol[b]], pair_rcp(sa[A0.bcol[b]] + mu)) : xz<E>();
        T ww = 0, den = 0;
        E s[NB1];
#pragma unroll
        for (int r = 0; r < NB; ++r) s[r] = xz<E>();
        for (int c = sl; c < W; c += rs) {
            const int t = CPLX ? hx_t(c, n, W) : c;
            const bool pair = CPLX && !hx_self(c, n, W);
            const T wg = pair ? (T)2 : (T)1;
            const T s0 = pair_rcp(sa[c] + mu);
            const E P0 = xs(sg[c], s0);
            den += wg * s0;
#pragma unroll
            for (int r = 0; r < NB; ++r)
                if (r < nb) {
                    s[r] = xa(s[r], xm(V0[(size_t)r * n + t], P0));
                    if (pair) s[r] = xa(s[r], xm(V0[(size_t)r * n + hx_neg(t, n)], xc(P0)));
                }
            if (t >= k && t < n - k) {
                E w = P0;
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    if (b < nb) w = xa(w, xm(b0[(size_t)b * A0.N + (t - k)], pb[b]));
                ww += wg * abs2_of(w);
            }
        }
        if (rs > 1) {
            ww = lane_sum(ww, rs);
            den = lane_sum(den, rs);
#pragma unroll
            for (int r = 0; r < NB; ++r) s[r] = lane_sum(s[r], rs);
        }
        T vsq = 0;
#pragma unroll
        for (int r = 0; r < NB; ++r)
            if (r < nb) vsq += abs2_of(s[r]);
        if (j < K && sl == 0) G[item * K + j] = ((double)ww + (double)vsq) / ((double)den * (double)den);
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
    cudaFree(x->s_idx); cudaFree(x->s_mu); cudaFree(x->s_G); cudaFree(x->s_best); cudaFree(x->red);
    delete x;
    p->exact = nullptr;
}

namespace {

int border_count(int fam) {
    if (fam == HOBC_FAMILY_SINE || fam == HOBC_FAMILY_COSINE || fam == HOBC_FAMILY_FOURIER) return 1;
    if (fam == HOBC_FAMILY_SINE_CUBIC || fam == HOBC_FAMILY_COSINE_QUARTIC) return 2;
    if (fam == HOBC_FAMILY_REFLECTIVE || fam == HOBC_FAMILY_PERIODIC) return 0;   // T orthogonal
    return -1;
}

// Builds the row split of each axis and the line-sum buffers on first use.
hobc_status ensure_exact(hobc_plan_s* p) {
    if (p->exact) return HOBC_OK;
    const int k = border_count(p->fam);
    if (k < 0) {
        set_last_error_text("hobc_gcv_exact: unsupported family");
        return HOBC_ERR_UNSUPPORTED;
    }
    hobc_exact_s* x = new hobc_exact_s();
    p->exact = x;
    x->k = k;
    x->cplx = p->fam == HOBC_FAMILY_FOURIER;
    const bool fp64 = p->prec == HOBC_FP64;
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < p->nax; ++a) {
        const int n = p->ax[a].n;
        x->N[a] = n - 2 * k;
        for (int b = 0; b < 2 * k; ++b) x->bidx[a][b] = b < k ? b : n - 2 * k + b;
        std::vector<cdx> bhat(1, cdx(0, 0)), V(1, cdx(0, 0));
        if (k > 0) {
            std::vector<cdx> Tm;
            hobc_status s = axis_matrix(p->fam, n, p->stream, Tm);
            if (s == HOBC_OK) s = split_rows(Tm, n, k, bhat, V);
            if (s != HOBC_OK) { exact_free(p); return s; }
        }
        if (e == cudaSuccess) e = fp64 ? upload<double>(&x->bhat[a], bhat, x->cplx) : upload<float>(&x->bhat[a], bhat, x->cplx);
        if (e == cudaSuccess) e = fp64 ? upload<double>(&x->V[a], V, x->cplx) : upload<float>(&x->V[a], V, x->cplx);
        if (e == cudaSuccess) e = upload<double>(&x->Vd[a], V, x->cplx);
    }
    const size_t B = (size_t)p->desc.batch, K = (size_t)p->K;
    if (p->nax == 2) {
        const size_t n0 = (size_t)p->ax[0].n, W1 = (size_t)p->ax[1].W;
        const size_t cv = 2 * (size_t)k * (x->cplx ? 2 : 1);
        if (e == cudaSuccess) e = cudaMalloc(&x->col_out, B * W1 * (2 + cv) * K * p->esz);
        if (e == cudaSuccess) e = cudaMalloc(&x->row_out, B * n0 * std::max(cv, (size_t)1) * K * p->esz);
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
    A.W = p->ax[a].W;
    for (int b = 0; b < 2 * x->k; ++b) {
        A.bidx[b] = x->bidx[a][b];
        A.bcol[b] = (x->cplx && a == p->nax - 1 && A.bidx[b] == A.n - 1) ? A.W - 1 : A.bidx[b];
    }
    return A;
}

// Lanes per grid value: one grid value per thread for K >= 256; for fewer
// values the lines are cut into rs slices (adjacent lanes, summed by
// butterflies) so that a CTA still runs 256 threads.
int lane_slices(int K) {
    int jp = 1;
    while (jp < K && jp < 256) jp *= 2;
    return std::min(32, std::max(1, 256 / jp));
}

// G_ex at Kp values of mu per problem (muT + item * mu_stride, plan
// precision) into Gout [batch][Kp].
template <typename T, bool CPLX, int NB>
hobc_status run_exact_pass(hobc_plan_s* p, const void* ghat, const void* D, const T* muT, int mu_stride, int Kp,
                           double* Gout) {
    typedef typename ElemT<T, CPLX>::t E;
    hobc_exact_s* x = p->exact;
    GcvGeom geo = exact_geo(p);
    geo.K = Kp;
    const int B = p->desc.batch;
    constexpr int k = NB / 2;
    const E* sp = reinterpret_cast<const E*>(ghat);
    const E* dp = reinterpret_cast<const E*>(D);
    const long long dps = (long long)p->spec_elems;
    const int rs = lane_slices(Kp);
    const int threads = rs > 1 ? 256 : std::min(256, (Kp + 31) / 32 * 32);
    const size_t el = sizeof(T) + sizeof(E);
    cudaError_t e = cudaSuccess;
    if (p->nax == 1) {
        const ExAxis A0 = ex_axis(x, p, 0);
        (rs > 1 ? k_ex_1d<T, CPLX, NB, true> : k_ex_1d<T, CPLX, NB, false>)<<<B, threads, (size_t)A0.W * el, p->stream>>>(sp, dp, dps, p->desc.psf_per_item, muT,
                                                                          mu_stride, rs, geo, A0, Gout);
        p->launches += 1;
    } else {
        const ExAxis A0 = ex_axis(x, p, 0), A1 = ex_axis(x, p, 1);
        const int n0 = A0.n, W1 = A1.W;
        const size_t sc = (size_t)(kExCB + 2 * k) * n0 * el, sr = (size_t)(CPLX ? 2 : 1) * W1 * el;
        auto cols = rs > 1 ? k_ex_cols<T, CPLX, NB, true> : k_ex_cols<T, CPLX, NB, false>;
        auto rows = rs > 1 ? k_ex_rows<T, CPLX, NB, true> : k_ex_rows<T, CPLX, NB, false>;
        e = cudaFuncSetAttribute(cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
        if (e != cudaSuccess) { set_last_error("hobc_gcv_exact", e); return HOBC_ERR_CUDA; }
        cols<<<dim3((unsigned)((W1 + kExCB - 1) / kExCB), (unsigned)B), threads, sc, p->stream>>>(
            sp, dp, dps, p->desc.psf_per_item, muT, mu_stride, rs, geo, A0, A1, reinterpret_cast<T*>(x->col_out));
        if (NB > 0)
            rows<<<dim3((unsigned)(CPLX ? (n0 - 2) / 2 + 3 : n0), (unsigned)B), threads, sr, p->stream>>>(
                sp, dp, dps, p->desc.psf_per_item, muT, mu_stride, rs, geo, A0, A1, reinterpret_cast<T*>(x->row_out));
        // lanes per grid value and line partitions so that the reduction keeps
        // the SMs busy however few values a pass evaluates
        int ls_log2 = 0;
        while ((32 >> (ls_log2 + 1)) >= Kp && ls_log2 < 5) ++ls_log2;
        const int jpc = 32 >> ls_log2;
        const int cy = (Kp + jpc - 1) / jpc;
        const int P = std::max(1, std::min(kExParts, (2 * 152 + B * cy - 1) / (B * cy)));
        constexpr int NV = 4 + 2 * (NB > 0 ? NB : 1) * (NB > 0 ? NB : 1);
        const size_t need = (size_t)B * P * Kp * NV;
        if (need > x->red_cap) {
            cudaFree(x->red);
            x->red = nullptr;
            x->red_cap = 0;
            e = cudaMalloc((void**)&x->red, need * sizeof(double));
            if (e != cudaSuccess) { set_last_error("hobc_gcv_exact (workspace)", e); return HOBC_ERR_CUDA; }
            x->red_cap = need;
        }
        k_ex_reduce<T, CPLX, NB><<<dim3((unsigned)B, (unsigned)cy, (unsigned)P), dim3(32, kExSlots), 0, p->stream>>>(
            reinterpret_cast<const T*>(x->col_out), reinterpret_cast<const T*>(x->row_out), A0, A1,
            reinterpret_cast<const double*>(x->Vd[1]), Kp, ls_log2, x->red);
        k_ex_finish<NB><<<B, std::min(256, (Kp + 31) / 32 * 32), 0, p->stream>>>(x->red, Kp, P, Gout);
        p->launches += NB > 0 ? 4 : 3;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error("hobc_gcv_exact", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

template <typename T, bool CPLX, int NB>
hobc_status run_gcv_exact(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    double* Gout = gcv ? gcv : p->exact->G;
    hobc_status s = run_exact_pass<T, CPLX, NB>(p, ghat, D, reinterpret_cast<const T*>(p->muT), 0, p->K, Gout);
    if (s != HOBC_OK) return s;
    k_ex_argmin<<<p->desc.batch, 256, 0, p->stream>>>(Gout, p->K, mu_idx);
    p->launches += 1;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error("hobc_gcv_exact", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

// ------------------------------------------------ coarse-to-fine search
// Three levels for 32 < K <= 1921, with s1 = ceil((K - 1) / 15) and
// s2 = min(s1, max(4, ceil(s1 / 8))): level 0 evaluates the grid values 0, s1,
// 2 s1, ... and K - 1 (at most 16); level 1 the incumbent +- s2 m, m = 1 ..
// ceil(s1 / s2) - 1; level 2 the incumbent +- 1 .. s2 - 1 (the incumbent: the
// first minimiser of every value evaluated so far; indices clamped into the
// grid).  Where G_ex is unimodal over the grid this reaches the grid's
// minimiser; at K = 256 after 16 + 8 + 6 evaluations.
constexpr int kExsSlots = 32;      // list slots per problem and level

__host__ __device__ inline bool exs_searched(int K) { return K > 32 && K <= 1921; }
__host__ __device__ inline int exs_s1(int K) { return (K - 1 + 14) / 15; }
__host__ __device__ inline int exs_s2(int K) {
    const int s1 = exs_s1(K), q = (s1 + 7) / 8;
    return s1 < (q > 4 ? q : 4) ? s1 : (q > 4 ? q : 4);
}
__host__ __device__ inline int exs_level_count(int level, int K) {
    const int s1 = exs_s1(K), s2 = exs_s2(K);
    if (level == 0) return (K - 1) / s1 + 1 + ((K - 1) % s1 != 0);
    if (level == 1) return 2 * ((s1 + s2 - 1) / s2 - 1);
    return 2 * (s2 - 1);
}

// The list of grid indices of one level (and their mu in plan precision).
template <typename T>
__global__ void k_exs_list(int level, int K, const T* __restrict__ muT, const int* __restrict__ best_idx,
                           int* __restrict__ idx, T* __restrict__ mu) {
    const long long item = blockIdx.x;
    const int n = exs_level_count(level, K);
    const int s1 = exs_s1(K), s2 = exs_s2(K);
    for (int j = threadIdx.x; j < kExsSlots; j += blockDim.x) {
        int k = 0;
        if (j < n) {
            if (level == 0) {
                k = j * s1 < K ? j * s1 : K - 1;
            } else {
                const int m = j / 2 + 1;                             // -m, +m in turn
                k = best_idx[item] + ((j & 1) ? 1 : -1) * m * (level == 1 ? s2 : 1);
                k = k < 0 ? 0 : (k > K - 1 ? K - 1 : k);
            }
        }
        idx[item * kExsSlots + j] = k;
        mu[item * kExsSlots + j] = muT[k];
    }
}

// Folds one level's values into each problem's incumbent (smaller G, or equal
// G at a smaller index; NaN never wins) and copies them into the curve.
// grid = items, block = 32.
__global__ void k_exs_pick(int level, int K, const double* __restrict__ Gl, const int* __restrict__ idx,
                           double* __restrict__ best_val, int* __restrict__ best_idx, double* __restrict__ curve) {
    const long long item = blockIdx.x;
    const int n = exs_level_count(level, K);
    const int j = threadIdx.x;
    double key = INFINITY;
    int bi = 0x7fffffff;
    if (j < n) {
        const double v = Gl[item * n + j];
        const int k = idx[item * kExsSlots + j];
        key = isnan(v) ? INFINITY : v;
        bi = k;
        if (curve) curve[item * K + k] = v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ok = __shfl_xor_sync(0xffffffffu, key, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ok < key || (ok == key && oi < bi)) { key = ok; bi = oi; }
    }
    if (j == 0) {
        double bv = level == 0 ? INFINITY : best_val[item];
        int bk = level == 0 ? 0x7fffffff : best_idx[item];
        if (key < bv || (key == bv && bi < bk)) { bv = key; bk = bi; }
        best_val[item] = bv;
        best_idx[item] = bk == 0x7fffffff ? 0 : bk;
    }
}

__global__ void k_exs_fill_nan(double* __restrict__ curve, long long count) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
        curve[i] = __longlong_as_double(0x7ff8000000000000LL);
}

template <typename T, bool CPLX, int NB>
hobc_status run_gcv_exact_search(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    const int B = p->desc.batch, K = p->K;
    if (!exs_searched(K)) return run_gcv_exact<T, CPLX, NB>(p, ghat, D, gcv, mu_idx);
    hobc_exact_s* x = p->exact;
    cudaError_t e = cudaSuccess;
    if (!x->s_idx) {
        e = cudaMalloc((void**)&x->s_idx, (size_t)B * kExsSlots * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&x->s_mu, (size_t)B * kExsSlots * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void**)&x->s_G, (size_t)B * kExsSlots * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void**)&x->s_best, (size_t)B * sizeof(double));
        if (e != cudaSuccess) { set_last_error("hobc_gcv_exact_search (workspace)", e); return HOBC_ERR_CUDA; }
    }
    if (gcv) {
        k_exs_fill_nan<<<std::min(1024, (B * K + 255) / 256), 256, 0, p->stream>>>(gcv, (long long)B * K);
        p->launches += 1;
    }
    T* smu = reinterpret_cast<T*>(x->s_mu);
    const T* muT = reinterpret_cast<const T*>(p->muT);
    for (int level = 0; level < 3; ++level) {
        const int n = exs_level_count(level, K);
        if (n == 0) continue;
        k_exs_list<T><<<B, 32, 0, p->stream>>>(level, K, muT, mu_idx, x->s_idx, smu);
        p->launches += 1;
        hobc_status s = run_exact_pass<T, CPLX, NB>(p, ghat, D, smu, kExsSlots, n, x->s_G);
        if (s != HOBC_OK) return s;
        k_exs_pick<<<B, 32, 0, p->stream>>>(level, K, x->s_G, x->s_idx, x->s_best, mu_idx, gcv);
        p->launches += 1;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error("hobc_gcv_exact_search", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

// Border vectors per axis: 2 (sine, cosine, Fourier), 4 (degree 3), 0 (orthogonal T).
template <typename T, bool SEARCH>
hobc_status gcv_exact_real(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    switch (p->exact->k) {
        case 0: return SEARCH ? run_gcv_exact_search<T, false, 0>(p, ghat, D, gcv, mu_idx)
                              : run_gcv_exact<T, false, 0>(p, ghat, D, gcv, mu_idx);
        case 2: return SEARCH ? run_gcv_exact_search<T, false, 4>(p, ghat, D, gcv, mu_idx)
                              : run_gcv_exact<T, false, 4>(p, ghat, D, gcv, mu_idx);
        default: return SEARCH ? run_gcv_exact_search<T, false, 2>(p, ghat, D, gcv, mu_idx)
                               : run_gcv_exact<T, false, 2>(p, ghat, D, gcv, mu_idx);
    }
}

template <bool SEARCH>
hobc_status gcv_exact_dispatch(hobc_plan_s* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    const bool F = p->exact->cplx;
    if (p->prec == HOBC_FP64) {
        if (F) return SEARCH ? run_gcv_exact_search<double, true, 2>(p, ghat, D, gcv, mu_idx)
                             : run_gcv_exact<double, true, 2>(p, ghat, D, gcv, mu_idx);
        return gcv_exact_real<double, SEARCH>(p, ghat, D, gcv, mu_idx);
    }
    if (F) return SEARCH ? run_gcv_exact_search<float, true, 2>(p, ghat, D, gcv, mu_idx)
                         : run_gcv_exact<float, true, 2>(p, ghat, D, gcv, mu_idx);
    return gcv_exact_real<float, SEARCH>(p, ghat, D, gcv, mu_idx);
}

}  // namespace
}  // namespace hobc

using namespace hobc;

namespace {
template <bool SEARCH>
hobc_status deblur_exact_impl(hobc_plan* p, const void* g_dev, const void* psf_dev, void* f_dev, int* mu_index_dev,
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
    if (s == HOBC_OK) s = gcv_exact_dispatch<SEARCH>(p, p->G, p->D, gcv_dev, mi);
    if (s == HOBC_OK)
        s = fp64 ? run_filter_synthesis<double>(p, p->G, p->D, mi, f_dev)
                 : run_filter_synthesis<float>(p, p->G, p->D, mi, f_dev);
    return s;
}
}  // namespace

extern "C" {

hobc_status hobc_gcv_exact(hobc_plan* p, const void* ghat_dev, const void* d_dev, double* gcv_dev, int* mu_index_dev) {
    if (!p || !ghat_dev || !d_dev || !mu_index_dev) return HOBC_ERR_ARG;
    hobc_status s = ensure_exact(p);
    if (s != HOBC_OK) return s;
    p->launches = 0;
    return gcv_exact_dispatch<false>(p, ghat_dev, d_dev, gcv_dev, mu_index_dev);
}

hobc_status hobc_gcv_exact_search(hobc_plan* p, const void* ghat_dev, const void* d_dev, double* gcv_dev,
                                  int* mu_index_dev) {
    if (!p || !ghat_dev || !d_dev || !mu_index_dev) return HOBC_ERR_ARG;
    hobc_status s = ensure_exact(p);
    if (s != HOBC_OK) return s;
    p->launches = 0;
    return gcv_exact_dispatch<true>(p, ghat_dev, d_dev, gcv_dev, mu_index_dev);
}


hobc_status hobc_deblur_exact(hobc_plan* p, const void* g_dev, const void* psf_dev, void* f_dev, int* mu_index_dev,
                              double* gcv_dev) {
    return deblur_exact_impl<false>(p, g_dev, psf_dev, f_dev, mu_index_dev, gcv_dev);
}

hobc_status hobc_deblur_exact_search(hobc_plan* p, const void* g_dev, const void* psf_dev, void* f_dev,
                                     int* mu_index_dev, double* gcv_dev) {
    return deblur_exact_impl<true>(p, g_dev, psf_dev, f_dev, mu_index_dev, gcv_dev);
}

}  // extern "C"
