// C ABI of the library (include/hobc.h): plan creation with the per-axis
// tables of the high-order boundary-condition transforms, workspace, and the
// entry points that run the hot path on the plan's stream.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "hobc_internal.h"
#include "hobc_device.cuh"
#include "hobc_kernels.cuh"

using hobc::AxisHost;
typedef std::complex<double> cd;

namespace hobc {

static thread_local char g_last_error[512] = "";

void set_last_error(const char* what, cudaError_t e) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

void set_last_error_text(const char* text) { snprintf(g_last_error, sizeof(g_last_error), "%s", text); }

// ------------------------------------------------------------- GCV finalize

// One cluster of nblk CTAs per problem.  A CTA owns the grid values
// j = rank*32 + lane (+ nblk*32 per further stripe); its 8 warps sum the chunk
// partials c = warp, warp + 8, ... of those values in double, the 8 slice sums
// are added in slice order, and G = num / den^2 is formed.  Each CTA keeps its
// first minimum (NaN never wins) in shared memory, and rank 0 combines the
// cluster's minima through distributed shared memory.  The order of every sum
// is fixed, so results do not depend on scheduling.
constexpr int kFinJ = 32, kFinSlices = 8, kFinMaxCluster = 8;

__global__ void __launch_bounds__(kFinJ * kFinSlices)
k_gcv_finalize(const double* __restrict__ partials, int nchunks, int K, double* __restrict__ gcv,
               int* __restrict__ mu_idx) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int nblk = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    __shared__ double sn[kFinSlices][kFinJ], sd[kFinSlices][kFinJ];
    __shared__ double best_v;
    __shared__ int best_i;
    const long long item = blockIdx.x / nblk;
    const double* p = partials + item * (long long)nchunks * 2 * K;
    const int lane = threadIdx.x % kFinJ, slice = threadIdx.x / kFinJ;
    double best = INFINITY;
    int bi = 0x7fffffff;
    for (int jb = rank * kFinJ; jb < K; jb += nblk * kFinJ) {
        const int j = jb + lane;
        double num = 0, den = 0;
        if (j < K)
            for (int c = slice; c < nchunks; c += kFinSlices) {
                num += p[(long long)c * 2 * K + j];
                den += p[(long long)c * 2 * K + K + j];
            }
        sn[slice][lane] = num;
        sd[slice][lane] = den;
        __syncthreads();
        if (slice == 0 && j < K) {
            num = 0;
            den = 0;
#pragma unroll
            for (int s = 0; s < kFinSlices; ++s) { num += sn[s][lane]; den += sd[s][lane]; }
            const double G = num / (den * den);
            if (gcv) gcv[item * K + j] = G;
            const double key = isnan(G) ? INFINITY : G;
            if (key < best || (key == best && j < bi)) { best = key; bi = j; }
        }
        __syncthreads();
    }
    if (slice == 0) {
        for (int off = 16; off > 0; off >>= 1) {
            const double v2 = __shfl_down_sync(0xffffffffu, best, off);
            const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
            if (v2 < best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
        }
        if (lane == 0) { best_v = best; best_i = bi; }
    }
    cluster.sync();
    if (rank == 0 && threadIdx.x == 0) {
        double v = INFINITY;
        int i = 0x7fffffff;
        for (int r = 0; r < nblk; ++r) {
            const double v2 = *cluster.map_shared_rank(&best_v, r);
            const int i2 = *cluster.map_shared_rank(&best_i, r);
            if (v2 < v || (v2 == v && i2 < i)) { v = v2; i = i2; }
        }
        mu_idx[item] = i == 0x7fffffff ? 0 : i;
    }
    cluster.sync();      // the other CTAs' shared memory stays valid until rank 0 has read it
}

cudaError_t launch_gcv_finalize_raw(const double* partials, int nchunks, int K, int batch, double* gcv,
                                    int* mu_idx, cudaStream_t st) {
    const int nblk = std::min(kFinMaxCluster, (K + kFinJ - 1) / kFinJ);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((long long)batch * nblk));
    cfg.blockDim = dim3(kFinJ * kFinSlices);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)nblk;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_gcv_finalize, partials, nchunks, K, gcv, mu_idx);
}

hobc_status launch_gcv_finalize(hobc_plan_s* p, double* gcv, int* mu_idx) {
    cudaError_t e = launch_gcv_finalize_raw(p->partials, p->gcv_chunks, p->K, p->desc.batch, gcv, mu_idx, p->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error("k_gcv_finalize", e);
        return HOBC_ERR_CUDA;
    }
    ++p->launches;
    return HOBC_OK;
}

// ------------------------------------------------------------------ tables

static void fft_host(std::vector<cd>& a) {   // in-place radix-2, exp(-i ...)
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        for (size_t i = 0; i < n; i += len) {
            for (size_t k = 0; k < len / 2; ++k) {
                const double ang = -2.0 * M_PI * (double)k / (double)len;
                const cd w(cos(ang), sin(ang));
                const cd u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}

// exp(-i pi a/b) with the argument reduced exactly (a may be negative).
cd expm_ipi(long long a, long long b) {
    long long r = a % (2 * b);
    if (r < 0) r += 2 * b;
    const double ang = M_PI * (double)r / (double)b;
    return cd(cos(ang), -sin(ang));
}

// theta/pi of spectral index t as the fraction num/den (border columns: 0).
void theta_frac(int fam, int n, int t, long long& num, long long& den) {
    const int N = n - 2;
    if (fam == hobc::FAM_R) { num = t; den = n; return; }          // comparison families: no border columns
    if (fam == hobc::FAM_PH || fam == hobc::FAM_P) { num = 2LL * t; den = n; return; }
    if (t == 0 || t == n - 1) { num = 0; den = 1; return; }
    if (fam == hobc::FAM_F4) {                     // degree 4, Fourier basis: DFT of order n - 4
        if (t == 1 || t == n - 2) { num = 0; den = 1; }
        else { num = 2LL * (t - 2); den = n - 4; }
        return;
    }
    if (fam == hobc::FAM_S3) {                     // N of the cubic family is n - 4
        if (t == 1 || t == n - 2) { num = 0; den = 1; }
        else { num = t - 1; den = n - 3; }
        return;
    }
    if (fam == hobc::FAM_C4) {                     // degree 4: DCT-II of order n - 4
        if (t == 1 || t == n - 2) { num = 0; den = 1; }
        else { num = t - 2; den = n - 4; }
        return;
    }
    if (fam == hobc::FAM_S) { num = t; den = N + 1; }
    else if (fam == hobc::FAM_C) { num = t - 1; den = N; }
    else { num = 2 * (t - 1); den = N; }
}

// Left border column of T_X: p of Eq. (eq:ART) with unit norm (S); q on the
// grid of Eq. (eq:points)/(eq:ints) (C) or Eq. (eq:pointn)/(eq:intn) (F).
static std::vector<double> border_column(int fam, int n) {
    std::vector<double> v(n);
    for (int i = 0; i < n; ++i) {
        if (fam == hobc::FAM_S) {
            v[i] = 1.0 - (double)i / (double)(n - 1);
        } else if (fam == hobc::FAM_C) {
            const double x = (2.0 * i - 1.0) * M_PI / (2.0 * n - 4.0);
            const double b = (2.0 * n - 3.0) * M_PI / (2.0 * n - 4.0);
            v[i] = (b - x) * (b - x);
        } else {
            const double x = (i - 1.0) * 2.0 * M_PI / (n - 2.0);
            const double b = 2.0 * M_PI;
            v[i] = (b - x) * (b - x);
        }
    }
    double nrm = 0;
    for (double x : v) nrm += x * x;
    nrm = sqrt(nrm);
    for (double& x : v) x /= nrm;
    return v;
}

// Border columns L1, L2 of the cubic family on x_a = (a - 1) pi/(N+1),
// a = 0..n-1, N = n - 4: L1 = (x_{N+1} - x)(x_{N+2} - x), L2 = L1 (x_{N+2} - x),
// each of unit norm.
static void cubic_columns(int n, std::vector<double>& L1, std::vector<double>& L2) {
    const int N = n - 4;
    const double xa = M_PI, xb = (N + 2) * M_PI / (N + 1);
    L1.assign(n, 0.0);
    L2.assign(n, 0.0);
    double n1 = 0, n2 = 0;
    for (int a = 0; a < n; ++a) {
        const double x = (a - 1) * M_PI / (N + 1);
        L1[a] = (xa - x) * (xb - x);
        L2[a] = L1[a] * (xb - x);
        n1 += L1[a] * L1[a];
        n2 += L2[a] * L2[a];
    }
    for (int a = 0; a < n; ++a) { L1[a] /= sqrt(n1); L2[a] /= sqrt(n2); }
}

// Border columns Q1, Q2 of the degree-4 cosine family on x_a = (2a - 3) pi/(2N),
// a = 0..n-1, N = n - 4, b = x_{n-1}: Q1 = (b - x)^2, Q2 = (b - x)^4, each of
// unit norm.
static void quartic_columns(int n, std::vector<double>& Q1, std::vector<double>& Q2) {
    const int N = n - 4;
    const double b = (2.0 * (n - 1) - 3.0) * M_PI / (2.0 * N);
    Q1.assign(n, 0.0);
    Q2.assign(n, 0.0);
    double n1 = 0, n2 = 0;
    for (int a = 0; a < n; ++a) {
        const double x = (2.0 * a - 3.0) * M_PI / (2.0 * N);
        const double u = (b - x) * (b - x);
        Q1[a] = u;
        Q2[a] = u * u;
        n1 += Q1[a] * Q1[a];
        n2 += Q2[a] * Q2[a];
    }
    for (int a = 0; a < n; ++a) { Q1[a] /= sqrt(n1); Q2[a] /= sqrt(n2); }
}

// Border columns Q1, Q2 of the degree-4 Fourier family (reading R17) on
// x_a = (a - 2) 2 pi/N, a = 0..n-1, N = n - 4, b = x_{n-1}: Q1 = (b - x)^2,
// Q2 = (b - x)^4, each of unit norm.
static void fourier_quartic_columns(int n, std::vector<double>& Q1, std::vector<double>& Q2) {
    const int N = n - 4;
    const double b = (n - 3.0) * 2.0 * M_PI / N;
    Q1.assign(n, 0.0);
    Q2.assign(n, 0.0);
    double n1 = 0, n2 = 0;
    for (int a = 0; a < n; ++a) {
        const double x = (a - 2.0) * 2.0 * M_PI / N;
        const double u = (b - x) * (b - x);
        Q1[a] = u;
        Q2[a] = u * u;
        n1 += Q1[a] * Q1[a];
        n2 += Q2[a] * Q2[a];
    }
    for (int a = 0; a < n; ++a) { Q1[a] /= sqrt(n1); Q2[a] /= sqrt(n2); }
}

// Gauss-Jordan inverse of a 4x4 matrix with partial pivoting; false if singular.
static bool invert4(const double* A, double* inv) {
    double m[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) m[i][j] = j < 4 ? A[4 * i + j] : (j - 4 == i ? 1.0 : 0.0);
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(m[r][c]) > fabs(m[piv][c])) piv = r;
        if (m[piv][c] == 0.0) return false;
        for (int j = 0; j < 8; ++j) std::swap(m[c][j], m[piv][j]);
        const double d = m[c][c];
        for (int j = 0; j < 8; ++j) m[c][j] /= d;
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            const double f = m[r][c];
            for (int j = 0; j < 8; ++j) m[r][j] -= f * m[c][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) inv[4 * i + j] = m[i][j + 4];
    return true;
}

template <typename T>
static void* upload_complex(const std::vector<cd>& h, cudaError_t& err) {
    std::vector<T> tmp(2 * h.size());
    for (size_t i = 0; i < h.size(); ++i) { tmp[2 * i] = (T)h[i].real(); tmp[2 * i + 1] = (T)h[i].imag(); }
    void* d = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&d, tmp.size() * sizeof(T));
    if (err == cudaSuccess) err = cudaMemcpy(d, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice);
    return d;
}

template <typename T>
static void* upload_real(const std::vector<double>& h, cudaError_t& err) {
    std::vector<T> tmp(h.begin(), h.end());
    void* d = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&d, tmp.size() * sizeof(T));
    if (err == cudaSuccess) err = cudaMemcpy(d, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice);
    return d;
}

// Power-of-two FFT length M of a line of n samples of a family (the core DFT
// of length L = N, or 2(N + 1) for the sine families, padded for Bluestein).
static int order_of(int fam, int n) {
    return fam == FAM_P ? n : fam_nb(fam) == 2 ? n - 4 : n - 2;
}

int fft_length_of(int fam, int n) {
    const int N = order_of(fam, n);
    const int L = (fam == FAM_S || fam == FAM_S3) ? 2 * (N + 1) : N;
    if (L >= 8 && (L & (L - 1)) == 0) return L;
    int M = 8;
    while (M < 2 * L - 1) M *= 2;
    return M;
}

template <typename T>
cudaError_t build_axis_host(AxisHost& a, int fam, int n, int p, bool half, int radix) {
    memset(&a, 0, sizeof(a));
    a.fam = fam;
    a.n = n;
    a.p = p;
    a.sslot = -1;
    cudaError_t err = cudaSuccess;
    if (fam == hobc::FAM_R || fam == hobc::FAM_PH) {
        // the classical comparison conditions run only in the dense mode: no
        // FFT or border tables, only the grid and the eigen-exponential table
        a.N = n; a.L = n; a.M = 8; a.log2M = 3; a.tpg = 1; a.H = n; a.W = n;
    } else {
    a.N = order_of(fam, n);
    const int N = a.N;
    a.L = (fam == hobc::FAM_S || fam == hobc::FAM_S3) ? 2 * (N + 1) : N;
    if (a.L >= 8 && (a.L & (a.L - 1)) == 0) {
        a.M = a.L;
        a.blue = 0;
    } else {
        a.M = 8;
        while (a.M < 2 * a.L - 1) a.M *= 2;
        a.blue = 1;
    }
    a.log2M = 0;
    while ((1 << a.log2M) < a.M) ++a.log2M;
    const bool can16 = a.M >= 256 && a.log2M <= 12;
    a.r16 = radix == 0 ? (hobc::fft_r16(a.M) && can16) : (radix == 16 && can16);
    a.tpg = a.r16 ? a.M / 16 : a.M / 8;
    a.H = fam_fourier(fam) ? N / 2 + 1 : N;
    a.W = (fam_fourier(fam) && half) ? a.H + 2 * fam_nb(fam) : n;
    // The pair kernels' two stage rows of a group fit in its own buffer above the
    // slots their FFT input and output occupy (positions < L) and below the
    // border-coefficient slots (M + M/16): with the chirp-z padding (M >= 2L - 1)
    // and for the sine families that is always so, and the CTA then needs no
    // separate stage (more of the SM's unified memory stays L1 for the tables).
    {
        const int esz_e = (fam_fourier(fam) ? 2 : 1) * (int)sizeof(T);
        const int need = (2 * a.W * esz_e + 2 * (int)sizeof(T) - 1) / (2 * (int)sizeof(T));
        const int first = (a.L - 1) + ((a.L - 1) >> 4) + 1;
        a.sslot = first + need <= a.M + a.M / 16 ? first : -1;
    }

    // per-stage twiddle tables in the order the FFT runs its stages: radix 16
    // while four or more bits remain (fft_r16) or radix 8 while three remain,
    // then one smaller radix; a stage with Ns > 1 stores W_{Ns R}^{pw k} =
    // W_M^{pw (M / (Ns R)) k}, k < Ns, for pw = 1, 2, 3, 4, 8, 12 (radix 16)
    // or pw = 1, 2, 4 (those < R)
    std::vector<cd> tw;
    const int rmax = a.r16 ? 16 : 8;
    for (int Ns = 1, rem = a.log2M; rem > 0;) {
        const int R = (1 << rem) >= rmax ? rmax : (1 << rem);
        std::vector<int> pws;
        if (R == 16) pws = {1, 2, 3, 4, 8, 12};
        else for (int pw = 1; pw < R; pw *= 2) pws.push_back(pw);
        if (Ns > 1)
            for (int pw : pws)
                for (int k = 0; k < Ns; ++k) tw.push_back(expm_ipi(2LL * pw * (a.M / (Ns * R)) * k, a.M));
        Ns *= R;
        rem -= R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1;
    }
    if (tw.empty()) tw.push_back(cd(1, 0));
    a.tw = upload_complex<T>(tw, err);
    if (a.blue) {
        std::vector<cd> chirp(a.L), c(a.M, cd(0, 0));
        for (long long k = 0; k < a.L; ++k) chirp[k] = expm_ipi((k * k) % (2LL * a.L), a.L);
        for (int m = 0; m < a.L; ++m) c[m] = std::conj(chirp[m]);
        for (int m = 1; m < a.L; ++m) c[a.M - m] = std::conj(chirp[m]);
        fft_host(c);
        for (cd& x : c) x /= (double)a.M;
        a.chirp = upload_complex<T>(chirp, err);
        a.bhat = upload_complex<T>(c, err);
    }
    if (fam == hobc::FAM_C || fam == hobc::FAM_C4) {
        std::vector<cd> post(N);
        for (int k = 0; k < N; ++k) post[k] = expm_ipi(k, 2LL * N);
        a.post = upload_complex<T>(post, err);
    }
    std::vector<double> q;
    if (fam == hobc::FAM_S3) {
        std::vector<double> L2;
        cubic_columns(n, q, L2);
        a.q2 = upload_real<T>(L2, err);
        // rows 0+2, 1, n-2, n-1+n-3 of T restricted to the border columns
        // (L1, L2, flip L2, flip L1)
        auto B = [&](int b, int r) {
            return b == 0 ? q[r] : b == 1 ? L2[r] : b == 2 ? L2[n - 1 - r] : q[n - 1 - r];
        };
        double K[16];
        for (int b = 0; b < 4; ++b) {
            K[0 * 4 + b] = B(b, 0) + B(b, 2);
            K[1 * 4 + b] = B(b, 1);
            K[2 * 4 + b] = B(b, n - 2);
            K[3 * 4 + b] = B(b, n - 1) + B(b, n - 3);
        }
        if (!invert4(K, a.k4) && err == cudaSuccess) err = cudaErrorInvalidValue;
    } else if (fam == hobc::FAM_F4) {
        std::vector<double> Q2;
        fourier_quartic_columns(n, q, Q2);
        a.q2 = upload_real<T>(Q2, err);
        // rows 0-(n-4), 1-(n-3), (n-2)-2, (n-1)-3 of T restricted to the border
        // columns (Q1, Q2, flip Q2, flip Q1): the periodic wrap cancels the
        // Fourier columns in these differences
        auto B = [&](int b, int r) {
            return b == 0 ? q[r] : b == 1 ? Q2[r] : b == 2 ? Q2[n - 1 - r] : q[n - 1 - r];
        };
        double K[16];
        for (int b = 0; b < 4; ++b) {
            K[0 * 4 + b] = B(b, 0) - B(b, n - 4);
            K[1 * 4 + b] = B(b, 1) - B(b, n - 3);
            K[2 * 4 + b] = B(b, n - 2) - B(b, 2);
            K[3 * 4 + b] = B(b, n - 1) - B(b, 3);
        }
        if (!invert4(K, a.k4) && err == cudaSuccess) err = cudaErrorInvalidValue;
    } else if (fam == hobc::FAM_P) {
        q.assign(n, 0.0);                    // periodic: no border columns
    } else if (fam == hobc::FAM_C4) {
        std::vector<double> Q2;
        quartic_columns(n, q, Q2);
        a.q2 = upload_real<T>(Q2, err);
        // rows 0-3, 1-2, (n-2)-(n-3), (n-1)-(n-4) of T restricted to the border
        // columns (Q1, Q2, flip Q2, flip Q1): the half-sample reflection cancels
        // the cosine columns in these differences
        auto B = [&](int b, int r) {
            return b == 0 ? q[r] : b == 1 ? Q2[r] : b == 2 ? Q2[n - 1 - r] : q[n - 1 - r];
        };
        double K[16];
        for (int b = 0; b < 4; ++b) {
            K[0 * 4 + b] = B(b, 0) - B(b, 3);
            K[1 * 4 + b] = B(b, 1) - B(b, 2);
            K[2 * 4 + b] = B(b, n - 2) - B(b, n - 3);
            K[3 * 4 + b] = B(b, n - 1) - B(b, n - 4);
        }
        if (!invert4(K, a.k4) && err == cudaSuccess) err = cudaErrorInvalidValue;
    } else {
        q = border_column(fam, n);
    }
    a.q = upload_real<T>(q, err);
    a.q1 = q[0];
    if (fam == hobc::FAM_C4 || fam == hobc::FAM_F4 || fam == hobc::FAM_P) {   // 4x4 solve, or none
        a.ka = 0.0;
        a.kb = 0.0;
    } else if (fam == hobc::FAM_S || fam == hobc::FAM_S3) {
        a.ka = 1.0 / q[0];
        a.kb = 0.0;
    } else {
        const double al = fam == hobc::FAM_C ? q[0] - q[1] : q[0] - q[n - 2];
        const double be = fam == hobc::FAM_C ? -q[n - 2] : -q[1];
        const double det = al * al - be * be;
        a.ka = al / det;
        a.kb = -be / det;
    }
    a.sc = fam_fourier(fam) ? 1.0 / sqrt((double)N) : sqrt(2.0 / (N + 1)) / 2.0;
    a.s0 = sqrt(1.0 / N);
    a.s1 = sqrt(2.0 / N);
    a.is0 = sqrt((double)N);
    a.is1 = sqrt(N / 2.0);
    a.invN = 1.0 / N;
    }
    // eigen-exponential table E[t][j] = exp(-i (j - m) theta_t), plus a unit entry
    const int m = p / 2;
    std::vector<double> et(2 * ((size_t)a.W * p + 1));
    for (int ts = 0; ts < a.W; ++ts) {
        const int t = (fam_fourier(fam) && half && ts >= a.W - fam_nb(fam)) ? n - (a.W - ts) : ts;
        long long num, den;
        theta_frac(fam, n, t, num, den);
        for (int j = 0; j < p; ++j) {
            const cd e = expm_ipi((long long)(j - m) * num, den);
            et[2 * ((size_t)ts * p + j)] = e.real();
            et[2 * ((size_t)ts * p + j) + 1] = e.imag();
        }
    }
    et[2 * (size_t)a.W * p] = 1.0;
    et[2 * (size_t)a.W * p + 1] = 0.0;
    if (err == cudaSuccess) err = cudaMalloc((void**)&a.etab, et.size() * sizeof(double));
    if (err == cudaSuccess) err = cudaMemcpy(a.etab, et.data(), et.size() * sizeof(double), cudaMemcpyHostToDevice);
    // float-float split of the same table (FP32 eigenvalue sums): x = hi + lo
    std::vector<float4> et2(et.size() / 2);
    for (size_t i = 0; i < et2.size(); ++i) {
        const float rh = (float)et[2 * i], ih = (float)et[2 * i + 1];
        et2[i] = make_float4(rh, (float)(et[2 * i] - (double)rh), ih, (float)(et[2 * i + 1] - (double)ih));
    }
    if (err == cudaSuccess) err = cudaMalloc((void**)&a.etab2, et2.size() * sizeof(float4));
    if (err == cudaSuccess)
        err = cudaMemcpy(a.etab2, et2.data(), et2.size() * sizeof(float4), cudaMemcpyHostToDevice);
    return err;
}

template cudaError_t build_axis_host<float>(AxisHost&, int, int, int, bool, int);
template cudaError_t build_axis_host<double>(AxisHost&, int, int, int, bool, int);

void free_axis(AxisHost& a) {
    cudaFree(a.tw); cudaFree(a.chirp); cudaFree(a.bhat); cudaFree(a.post); cudaFree(a.q); cudaFree(a.q2);
    cudaFree(a.etab);
    cudaFree(a.etab2);
    memset(&a, 0, sizeof(a));
}

// Checks the parts of a plan description that fix the geometry, the family and
// the precision, and resolves HOBC_FAMILY_AUTO.  check_psf: the PSF extents are
// part of the request (plans) or ignored (the allocation-free scan).
hobc_status resolve_desc(const hobc_plan_desc& d, bool check_psf, int* fam_out) {
    if (d.ndim != 1 && d.ndim != 2) return HOBC_ERR_ARG;
    if (d.n_mu < 1 || d.batch < 1) return HOBC_ERR_ARG;
    if (d.ndim == 2 && d.batch > 65535) return HOBC_ERR_SIZE;     // items ride on gridDim.y
    if (d.prec != HOBC_FP64 && d.prec != HOBC_FP32 && d.prec != HOBC_SPLIT_BF16) return HOBC_ERR_ARG;
    if (d.L != HOBC_L_IDENTITY && d.L != HOBC_L_LAPLACIAN) return HOBC_ERR_ARG;
    if (d.psf_per_item != 0 && d.psf_per_item != 1) return HOBC_ERR_ARG;
    for (int i = 0; i < d.ndim; ++i) {
        if (d.n[i] < 6 || d.n[i] > 1024) return HOBC_ERR_SIZE;
        if (!check_psf) continue;
        if (d.psf[i] < 1 || d.psf[i] % 2 == 0 || d.psf[i] > 63) return HOBC_ERR_SIZE;
        if (d.psf[i] > d.n[i] - 2) return HOBC_ERR_SIZE;       // 2m+1 <= n-2
    }
    const bool cubic = d.family == HOBC_FAMILY_SINE_CUBIC || d.family == HOBC_FAMILY_COSINE_QUARTIC ||
                       d.family == HOBC_FAMILY_FOURIER_QUARTIC ||
                       (d.family == HOBC_FAMILY_AUTO && (d.bc_degree == 3 || d.bc_degree == 4));
    if (cubic)
        for (int i = 0; i < d.ndim; ++i) {
            if (d.n[i] < 8) return HOBC_ERR_SIZE;                               // N = n-4 >= 4
            if (check_psf && d.psf[i] > d.n[i] - 4) return HOBC_ERR_SIZE;      // 2m+1 <= n-4
        }
    int fam = d.family;
    const bool comparison = fam == HOBC_FAMILY_REFLECTIVE || fam == HOBC_FAMILY_PERIODIC;
    if (fam == HOBC_FAMILY_PERIODIC && d.prec != HOBC_SPLIT_BF16) {
        // classical periodic conditions (Sec. 2, Eq. (eq:permat)) on the FFT path: the
        // DFT of order n, no border columns, any PSF
        if (d.bc_degree != 0) return HOBC_ERR_UNSUPPORTED;
        fam = FAM_P;
    } else if (comparison) {
        // classical conditions (Sec. 2): constants preserved, symmetric PSF; in the dense mode
        if (d.bc_degree != 0 || !d.psf_symmetric || d.prec != HOBC_SPLIT_BF16) return HOBC_ERR_UNSUPPORTED;
    } else {
        if (d.bc_degree < 1 || d.bc_degree > 4) return HOBC_ERR_UNSUPPORTED;
        if (fam == HOBC_FAMILY_AUTO) {
            if (d.bc_degree == 1) fam = d.psf_symmetric ? HOBC_FAMILY_SINE : -1;
            else if (d.bc_degree == 2) fam = d.psf_symmetric ? HOBC_FAMILY_COSINE : HOBC_FAMILY_FOURIER;
            else if (d.bc_degree == 3) fam = d.psf_symmetric ? HOBC_FAMILY_SINE_CUBIC : -1;
            else fam = d.psf_symmetric ? HOBC_FAMILY_COSINE_QUARTIC : HOBC_FAMILY_FOURIER_QUARTIC;
            if (fam < 0) return HOBC_ERR_UNSUPPORTED;   // sine families need a symmetric PSF (Sec. 2.2)
        }
        if (fam == HOBC_FAMILY_SINE && d.bc_degree != 1) return HOBC_ERR_UNSUPPORTED;
        if ((fam == HOBC_FAMILY_COSINE || fam == HOBC_FAMILY_FOURIER) && d.bc_degree != 2)
            return HOBC_ERR_UNSUPPORTED;
        if (fam == HOBC_FAMILY_SINE_CUBIC && d.bc_degree != 3) return HOBC_ERR_UNSUPPORTED;
        if (fam == HOBC_FAMILY_COSINE_QUARTIC && (d.bc_degree != 4 || !d.psf_symmetric))
            return HOBC_ERR_UNSUPPORTED;
        if (fam == HOBC_FAMILY_FOURIER_QUARTIC && d.bc_degree != 4) return HOBC_ERR_UNSUPPORTED;
        if (fam != HOBC_FAMILY_COSINE_QUARTIC && fam != HOBC_FAMILY_FOURIER_QUARTIC &&
            (fam < HOBC_FAMILY_SINE || fam > HOBC_FAMILY_SINE_CUBIC))
            return HOBC_ERR_ARG;
    }
    // degree 4 runs on the FFT path only (the dense engine has no matrices for it), and in
    // FP64 only: cond(T) is 644 already at n = 8 (7.5e4 at n = 32), so the FP32 rounding
    // bound 64 eps32 cond(T) exceeds 1e-3 at every size
    if ((fam == HOBC_FAMILY_COSINE_QUARTIC || fam == HOBC_FAMILY_FOURIER_QUARTIC) && d.prec != HOBC_FP64)
        return HOBC_ERR_UNSUPPORTED;
    *fam_out = fam;
    return HOBC_OK;
}

}  // namespace hobc

using namespace hobc;

// =================================================================== ABI

extern "C" {

const char* hobc_status_str(hobc_status s) {
    switch (s) {
        case HOBC_OK: return "HOBC_OK";
        case HOBC_ERR_ARG: return "HOBC_ERR_ARG";
        case HOBC_ERR_UNSUPPORTED: return "HOBC_ERR_UNSUPPORTED";
        case HOBC_ERR_SIZE: return "HOBC_ERR_SIZE";
        case HOBC_ERR_NONFINITE: return "HOBC_ERR_NONFINITE";
        case HOBC_ERR_CUDA: return "HOBC_ERR_CUDA";
        case HOBC_ERR_TIMEOUT: return "HOBC_ERR_TIMEOUT";
    }
    return "HOBC_ERR_UNKNOWN";
}

const char* hobc_last_error(void) { return g_last_error; }

void hobc_plan_destroy(hobc_plan* p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    for (int i = 0; i < 2; ++i)
        if (p->aux[i]) cudaStreamSynchronize(p->aux[i]);
    for (int i = 0; i < 2; ++i) free_axis(p->ax[i]);
    cudaFree(p->mu); cudaFree(p->muT); cudaFree(p->R); cudaFree(p->G); cudaFree(p->D);
    cudaFree(p->partials); cudaFree(p->gcv); cudaFree(p->mu_idx);
    cudaFree(p->g_in); cudaFree(p->f_out); cudaFree(p->psf_in);
    free_learned_ws(p);
    gcvx_free(p);
    dense_free(p);
    exact_free(p);
    for (int i = 0; i < 2; ++i)
        if (p->aux[i]) cudaStreamDestroy(p->aux[i]);
    for (int i = 0; i < 8; ++i) {
        if (p->ev_up[i]) cudaEventDestroy(p->ev_up[i]);
        if (p->ev_an[i]) cudaEventDestroy(p->ev_an[i]);
        if (p->ev_done[i]) cudaEventDestroy(p->ev_done[i]);
        if (p->ev_down[i]) cudaEventDestroy(p->ev_down[i]);
    }
    if (p->ev_psf) cudaEventDestroy(p->ev_psf);
    if (p->psf_pinned) cudaFreeHost(p->psf_pinned);
    delete p;
}

hobc_status hobc_plan_create(const hobc_plan_desc* desc, const double* mu_grid_host, void* cuda_stream,
                             hobc_plan** out) {
    if (!out) return HOBC_ERR_ARG;
    *out = nullptr;
    if (!desc || !mu_grid_host) return HOBC_ERR_ARG;
    const hobc_plan_desc d = *desc;
    int fam = 0;
    const hobc_status vs = resolve_desc(d, true, &fam);
    if (vs != HOBC_OK) return vs;
    for (int j = 0; j < d.n_mu; ++j) {
        if (!std::isfinite(mu_grid_host[j])) return HOBC_ERR_NONFINITE;
        if (!(mu_grid_host[j] > 0)) return HOBC_ERR_ARG;
        // FP32 GCV pairs grid values: (a + mu1)(a + mu2) must stay a normal float
        if (d.prec != HOBC_FP64 && (mu_grid_host[j] < 1e-18 || mu_grid_host[j] > 1e18)) return HOBC_ERR_ARG;
    }

    hobc_plan_s* p = new hobc_plan_s;
    memset(p, 0, sizeof(*p));
    p->desc = d;
    p->fam = fam;
    p->prec = d.prec;
    p->esz = d.prec == HOBC_FP64 ? 8 : 4;
    p->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    p->K = d.n_mu;
    p->nax = d.ndim;
    cudaGetDevice(&p->device);
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < d.ndim && err == cudaSuccess; ++i) {
        const bool half = (i == d.ndim - 1);
        err = d.prec == HOBC_FP64 ? build_axis_host<double>(p->ax[i], fam, d.n[i], d.psf[i], half)
                                  : build_axis_host<float>(p->ax[i], fam, d.n[i], d.psf[i], half);
    }
    const AxisHost& last = p->ax[d.ndim - 1];
    p->spec_elems = d.ndim == 1 ? (size_t)last.W : (size_t)last.W * p->ax[0].n;
    const size_t ebytes = p->esz * (fam_fourier(fam) ? 2 : 1);
    p->spec_bytes = p->spec_elems * ebytes;
    p->img_elems = d.ndim == 1 ? (size_t)d.n[0] : (size_t)d.n[0] * d.n[1];
    p->psf_elems = d.ndim == 1 ? (size_t)d.psf[0] : (size_t)d.psf[0] * d.psf[1];
    p->npsf = d.psf_per_item ? d.batch : 1;
    p->gcv_chunk = hobc::gcv_chunk_for((long long)p->spec_elems, p->K, d.prec == HOBC_FP64);
    p->gcv_chunks = (int)((p->spec_elems + p->gcv_chunk - 1) / p->gcv_chunk);
    const size_t B = (size_t)d.batch;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (err == cudaSuccess && bytes) err = cudaMalloc(ptr, bytes);
    };
    alloc((void**)&p->mu, sizeof(double) * p->K);
    alloc(&p->muT, p->esz * p->K);
    if (err == cudaSuccess) err = cudaMemcpy(p->mu, mu_grid_host, sizeof(double) * p->K, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) {
        if (d.prec == HOBC_FP64) {
            err = cudaMemcpy(p->muT, mu_grid_host, sizeof(double) * p->K, cudaMemcpyHostToDevice);
        } else {
            std::vector<float> mf(mu_grid_host, mu_grid_host + p->K);
            err = cudaMemcpy(p->muT, mf.data(), sizeof(float) * p->K, cudaMemcpyHostToDevice);
        }
    }
    if (d.ndim == 2) alloc(&p->R, B * p->spec_bytes);
    alloc(&p->G, B * p->spec_bytes);
    alloc(&p->D, (size_t)p->npsf * p->spec_bytes);
    alloc((void**)&p->partials, B * p->gcv_chunks * 2 * p->K * sizeof(double));
    alloc((void**)&p->gcv, B * p->K * sizeof(double));
    alloc((void**)&p->mu_idx, B * sizeof(int));
    alloc(&p->g_in, B * p->img_elems * p->esz);
    alloc(&p->f_out, B * p->img_elems * p->esz);
    alloc(&p->psf_in, (size_t)p->npsf * p->psf_elems * p->esz);
    if (err != cudaSuccess) {
        set_last_error("hobc_plan_create", err);
        hobc_plan_destroy(p);
        return HOBC_ERR_CUDA;
    }
    hobc_status s = d.prec == HOBC_FP64 ? prepare_kernels<double>(p) : prepare_kernels<float>(p);
    if (s == HOBC_OK && d.prec == HOBC_SPLIT_BF16) s = dense_prepare(p);
    if (s != HOBC_OK) {
        hobc_plan_destroy(p);
        return s;
    }
    *out = p;
    return HOBC_OK;
}

hobc_status hobc_plan_set_host_chunks(hobc_plan* p, int chunks) {
    if (!p || chunks < 0 || chunks > 8) return HOBC_ERR_ARG;
    // the per-chunk events order consecutive calls chunk by chunk: a new layout
    // starts from an idle plan
    cudaError_t e = p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize();
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        if (p->aux[i]) e = cudaStreamSynchronize(p->aux[i]);
    if (e != cudaSuccess) { set_last_error("hobc_plan_set_host_chunks", e); return HOBC_ERR_CUDA; }
    p->host_chunks = chunks;
    return HOBC_OK;
}

hobc_family hobc_plan_family(const hobc_plan* p) {
    if (!p) return HOBC_FAMILY_AUTO;
    return p->fam == FAM_P ? HOBC_FAMILY_PERIODIC : (hobc_family)p->fam;
}

int hobc_fft_length(int bc_degree, int n) {
    if (n < 8 || n > 1024) return 0;
    const int fam = bc_degree == 1 ? FAM_S : bc_degree == 2 ? FAM_C : bc_degree == 3 ? FAM_S3 : -1;
    return fam < 0 ? 0 : fft_length_of(fam, n);
}

hobc_status hobc_spectrum_size(const hobc_plan* p, size_t* spec, int* is_complex, size_t* psf) {
    if (!p) return HOBC_ERR_ARG;
    if (spec) *spec = p->spec_elems;
    if (is_complex) *is_complex = fam_fourier(p->fam);
    if (psf) *psf = p->psf_elems;
    return HOBC_OK;
}

int hobc_last_launch_count(const hobc_plan* p) { return p ? p->launches : 0; }

#define HOBC_DISPATCH(p, fn, ...) ((p)->prec == HOBC_FP64 ? fn<double>(p, __VA_ARGS__) : fn<float>(p, __VA_ARGS__))

hobc_status hobc_eigenvalues(hobc_plan* p, const void* psf, void* D) {
    if (!p || !psf || !D) return HOBC_ERR_ARG;
    p->launches = 0;
    return HOBC_DISPATCH(p, run_eig, psf, D);
}

hobc_status hobc_analysis(hobc_plan* p, const void* g, void* ghat) {
    if (!p || !g || !ghat) return HOBC_ERR_ARG;
    p->launches = 0;
    return HOBC_DISPATCH(p, run_analysis, g, ghat);
}

hobc_status hobc_synthesis(hobc_plan* p, const void* c, void* y) {
    if (!p || !c || !y) return HOBC_ERR_ARG;
    p->launches = 0;
    return HOBC_DISPATCH(p, run_synthesis, c, y);
}

hobc_status hobc_gcv(hobc_plan* p, const void* ghat, const void* D, double* gcv, int* mu_idx) {
    if (!p || !ghat || !D || !mu_idx) return HOBC_ERR_ARG;
    p->launches = 0;
    return HOBC_DISPATCH(p, run_gcv, ghat, D, gcv, mu_idx);
}

hobc_status hobc_filter_synthesis(hobc_plan* p, const void* ghat, const void* D, const int* mu_idx, void* f) {
    if (!p || !ghat || !D || !mu_idx || !f) return HOBC_ERR_ARG;
    p->launches = 0;
    return HOBC_DISPATCH(p, run_filter_synthesis, ghat, D, mu_idx, f);
}

static hobc_status deblur_impl(hobc_plan* p, const void* g, const void* psf, void* f, int* mu_idx, double* gcv) {
    int* mi = mu_idx ? mu_idx : p->mu_idx;
    hobc_status s = HOBC_DISPATCH(p, run_eig, psf, p->D);
    if (s == HOBC_OK) s = HOBC_DISPATCH(p, run_analysis, g, p->G);
    if (s == HOBC_OK) s = HOBC_DISPATCH(p, run_gcv, p->G, p->D, gcv, mi);
    if (s == HOBC_OK) s = HOBC_DISPATCH(p, run_filter_synthesis, p->G, p->D, mi, f);
    return s;
}

hobc_status hobc_deblur(hobc_plan* p, const void* g, const void* psf, void* f, int* mu_idx, double* gcv) {
    if (!p || !g || !psf || !f) return HOBC_ERR_ARG;
    if (g == f) return HOBC_ERR_ARG;
    p->launches = 0;
    return deblur_impl(p, g, psf, f, mu_idx, gcv);
}

// The plan seen as the sub-batch [c0, c0 + cb): per-item workspace offsets,
// its own stream.  A shallow copy: it owns nothing.
static hobc_plan_s chunk_view(const hobc_plan_s* p, size_t c0, size_t cb, cudaStream_t s) {
    hobc_plan_s v = *p;
    auto off = [&](void* base, size_t per_item) -> void* {
        return base ? static_cast<void*>(static_cast<char*>(base) + c0 * per_item) : nullptr;
    };
    v.desc.batch = (int)cb;
    v.stream = s;
    v.R = off(p->R, p->spec_bytes);
    v.G = off(p->G, p->spec_bytes);
    if (p->desc.psf_per_item) {
        v.D = off(p->D, p->spec_bytes);
        v.npsf = (int)cb;
    }
    v.partials = p->partials + c0 * (size_t)p->gcv_chunks * 2 * p->K;
    v.gcv = p->gcv + c0 * p->K;
    v.mu_idx = p->mu_idx + c0;
    v.g_in = off(p->g_in, p->img_elems * p->esz);
    v.f_out = off(p->f_out, p->img_elems * p->esz);
    v.item0 = p->item0 + c0;
    v.launches = 0;
    return v;
}

// Chunks of the host-buffer pipeline (at most the plan's 8 event pairs).  On
// 32 images of 1024^2, 4 chunks ran the call in 2.36 ms, 8 in 2.42, 2 in 2.60,
// 16 in 2.96: fewer chunks leave the first upload and the last download
// exposed, more run the kernels on grids too small to fill the GPU.
static const size_t kHostChunks = 4;

hobc_status hobc_deblur_host_async(hobc_plan* p, const void* g, const void* psf, void* f, int* mu_idx,
                                   double* gcv) {
    if (!p || !g || !psf || !f) return HOBC_ERR_ARG;
    p->launches = 0;
    const size_t B = (size_t)p->desc.batch;
    const size_t ib = p->img_elems * p->esz;
    const size_t pb = (size_t)p->npsf * p->psf_elems * p->esz;
    const size_t want = p->host_chunks > 0 ? (size_t)p->host_chunks : kHostChunks;
    const size_t nchunk = B >= want ? want : B;
    const size_t cb = (B + nchunk - 1) / nchunk;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        if (!p->aux[i]) e = cudaStreamCreateWithFlags(&p->aux[i], cudaStreamNonBlocking);
    for (size_t i = 0; i < nchunk && e == cudaSuccess; ++i) {
        cudaEvent_t* evs[4] = {&p->ev_up[i], &p->ev_an[i], &p->ev_done[i], &p->ev_down[i]};
        for (cudaEvent_t* ev : evs)
            if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    }
    if (e == cudaSuccess && !p->ev_psf) e = cudaEventCreateWithFlags(&p->ev_psf, cudaEventDisableTiming);
    if (e == cudaSuccess && !p->psf_pinned) e = cudaMallocHost(&p->psf_pinned, pb);
    // the PSF goes through page-locked staging (a copy from pageable memory
    // would wait for the plan's stream); the staging is rewritten once the
    // previous call's copy of it has left
    if (e == cudaSuccess) e = cudaEventSynchronize(p->ev_psf);
    if (e == cudaSuccess) {
        memcpy(p->psf_pinned, psf, pb);
        e = cudaMemcpyAsync(p->psf_in, p->psf_pinned, pb, cudaMemcpyHostToDevice, p->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_psf, p->stream);
    if (e != cudaSuccess) { set_last_error("hobc_deblur_host_async set-up", e); return HOBC_ERR_CUDA; }
    hobc_status s = HOBC_DISPATCH(p, run_eig, p->psf_in, p->D);
    if (s != HOBC_OK) return s;
    // the expansion's steps that depend on the eigenvalues alone run once per call
    const bool gx_once = gcvx_active(p) && p->nax == 2 && p->prec != HOBC_FP64;
    if (gx_once) {
        s = gcvx_prepare(p, p->D);
        if (s != HOBC_OK) return s;
    }
    // three-stage pipeline over chunks of the batch: every upload back to back
    // on aux[0], each chunk's kernels in order on the plan's stream once its
    // upload is done, each download on aux[1] once its kernels are done.
    // Across calls, a chunk's upload waits until the previous call's analysis
    // has read its input slots, and its filter + synthesis until the previous
    // call's download has read its output slots.
    for (size_t c0 = 0, c = 0; c0 < B && e == cudaSuccess; c0 += cb, ++c) {
        const size_t n = std::min(cb, B - c0);
        e = cudaStreamWaitEvent(p->aux[0], p->ev_an[c], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<char*>(p->g_in) + c0 * ib, static_cast<const char*>(g) + c0 * ib, n * ib,
                                cudaMemcpyHostToDevice, p->aux[0]);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_up[c], p->aux[0]);
    }
    for (size_t c0 = 0, c = 0; c0 < B && e == cudaSuccess && s == HOBC_OK; c0 += cb, ++c) {
        const size_t n = std::min(cb, B - c0);
        e = cudaStreamWaitEvent(p->stream, p->ev_up[c], 0);
        if (e != cudaSuccess) break;
        hobc_plan_s v = chunk_view(p, c0, n, p->stream);
        v.gx_prepared = gx_once ? 1 : 0;
        s = HOBC_DISPATCH(&v, run_analysis, v.g_in, v.G);
        if (s == HOBC_OK) e = cudaEventRecord(p->ev_an[c], p->stream);
        if (s == HOBC_OK && e == cudaSuccess) s = HOBC_DISPATCH(&v, run_gcv, v.G, v.D, gcv ? v.gcv : nullptr, v.mu_idx);
        if (s == HOBC_OK && e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->ev_down[c], 0);
        if (s == HOBC_OK && e == cudaSuccess)
            s = HOBC_DISPATCH(&v, run_filter_synthesis, v.G, v.D, v.mu_idx, v.f_out);
        p->launches += v.launches;
        if (s != HOBC_OK || e != cudaSuccess) break;
        e = cudaEventRecord(p->ev_done[c], p->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->aux[1], p->ev_done[c], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<char*>(f) + c0 * ib, v.f_out, n * ib, cudaMemcpyDeviceToHost, p->aux[1]);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_down[c], p->aux[1]);
    }
    // the small outputs go on the plan's stream, after the last scan and
    // before anything a later call queues there
    if (e == cudaSuccess && s == HOBC_OK) {
        if (mu_idx) e = cudaMemcpyAsync(mu_idx, p->mu_idx, B * sizeof(int), cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess && gcv)
            e = cudaMemcpyAsync(gcv, p->gcv, B * p->K * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    }
    if (s != HOBC_OK) return s;
    if (e != cudaSuccess) { set_last_error("hobc_deblur_host_async", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

hobc_status hobc_plan_wait(hobc_plan* p) {
    if (!p) return HOBC_ERR_ARG;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2; ++i)
        if (p->aux[i]) {
            const cudaError_t e2 = cudaStreamSynchronize(p->aux[i]);
            if (e == cudaSuccess) e = e2;
        }
    const cudaError_t e2 = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) { set_last_error("hobc_plan_wait", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

hobc_status hobc_deblur_host(hobc_plan* p, const void* g, const void* psf, void* f, int* mu_idx, double* gcv) {
    const hobc_status s = hobc_deblur_host_async(p, g, psf, f, mu_idx, gcv);
    if (!p) return s;
    const hobc_status w = hobc_plan_wait(p);
    return s != HOBC_OK ? s : w;
}

}  // extern "C"
