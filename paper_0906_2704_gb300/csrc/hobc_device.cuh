// Device building blocks for the line transforms of the high-order boundary
// condition method (Donatelli, arXiv:0906.2704):
//   * complex helpers on float2/double2;
//   * a shared-memory Stockham FFT of power-of-two length M run by one "group"
//     of threads, every group of the CTA in lock-step so __syncthreads() can be
//     used: M/16 threads holding 16 values each for M >= 256 (radix-16 stages,
//     then one smaller radix), M/8 threads holding 8 values below (radix 8);
//   * Bluestein's chirp-z form for lengths L that are not powers of two
//     (X_k = b_k sum_j (x_j b_j) conj(b_{k-j}), b_k = exp(-i pi k^2 / L)), so
//     the awkward orders N = n - 2 of the paper (1022 = 2*7*73 ...) need no
//     special radices;
//   * the 2x2 boundary solve that replaces the Sherman-Morrison-Woodbury step
//     of Thm. 1 (Sec. 3.3), and the angle grids of Eq. (eq:jcf), (eq:Ac), (eq:Af).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hobc {

// FAM_S..FAM_F4 have the values of hobc_family; FAM_P is the periodic family
// on the FFT path (HOBC_FAMILY_PERIODIC outside the dense mode), FAM_PH the same
// conditions in the Hartley basis of the dense mode.
enum { FAM_S = 1, FAM_C = 2, FAM_F = 3, FAM_S3 = 4, FAM_R = 5, FAM_PH = 6, FAM_C4 = 7, FAM_F4 = 8, FAM_P = 9 };

// Families with a complex spectrum (Fourier basis) and their border entries
// on each side of a line: F 1, F4 2, P none.
__host__ __device__ constexpr bool fam_fourier(int fam) { return fam == FAM_F || fam == FAM_F4 || fam == FAM_P; }
__host__ __device__ constexpr int fam_nb(int fam) {
    return (fam == FAM_S3 || fam == FAM_C4 || fam == FAM_F4) ? 2 : (fam == FAM_P || fam == FAM_R || fam == FAM_PH) ? 0 : 1;
}

template <typename T> struct V2;
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<double> { typedef double2 t; };
template <typename T> using C2 = typename V2<T>::t;

template <typename T> __device__ __forceinline__ C2<T> cmk(T x, T y) { C2<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return cmk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return cmk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
    return cmk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ C2<T> cconj(C2<T> a) { return cmk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ C2<T> cscale(C2<T> a, T s) { return cmk<T>(a.x * s, a.y * s); }
template <typename T> __device__ __forceinline__ T cabs2(C2<T> a) { return a.x * a.x + a.y * a.y; }

// One transform axis: the order-n transform T_X of the paper and the tables of
// its length-L complex DFT core.  Built on the host (hobc_api.cu), passed by value.
template <typename T>
struct Axis {
    int fam;        // FAM_*
    int n;          // field-of-view length on this axis
    int N;          // order of the trigonometric block: n - 2 (n - 4 for S3, C4, F4; n for P)
    int L;          // length of the complex DFT core: N (C, F, C4, F4, P) or 2(N+1) (S, S3)
    int M;          // power-of-two FFT length (== L when L is a power of two >= 8)
    int log2M;
    int blue;       // 1: Bluestein (M >= 2L-1), 0: direct
    int tpg;        // threads per group: M/16 with radix-16 stages (r16), else M/8
    int r16;        // 1: radix-16 stages (M >= 256, log2M <= 12), 0: radix 8
    int Mp;         // shared-memory slots per group: group_slots(M)
    int sslot;      // >= 0: the group's two stage rows of the pair kernels sit in its own
                    // buffer from this slot on (free while they are used); -1: after
                    // every group's buffer
    int H;          // Fourier families: floor(N/2)+1 stored frequencies; else N
    int W;          // spectrum entries stored on this axis: n, or H + 2 NB on a half axis of a
                    // Fourier family (NB border entries on each side)
    const C2<T>* tw;      // per-stage twiddle tables of the FFT, concatenated (< M entries)
    const C2<T>* chirp;   // [L] exp(-i pi (k^2 mod 2L) / L)
    const C2<T>* bhat;    // [M] FFT_M(conj-chirp, wrapped) / M
    const C2<T>* post;    // COSINE: [N] exp(-i pi k / (2N))
    const T* q;           // [n] left border column of T_X (p for S, q for C, F, L1 for S3, Q1 for C4, F4)
    const T* q2;          // S3, C4, F4: [n] second left border column (L2, Q2)
    double ka, kb;        // inverse of the 2x2 border system, [[ka, kb], [kb, ka]]
    double k4[16];        // S3, C4, F4: inverse of the 4x4 border system, row-major
    T q1;                 // q[0]
    T sc;                 // Fourier families: 1/sqrt(N); S, S3: sqrt(2/(N+1))/2
    T s0, s1;             // C: DCT-II row scales sqrt(1/N), sqrt(2/N)
    T is0, is1;           // C: their reciprocals
    T invN;               // C: 1/N
};

// ---------------------------------------------------------------- FFT core

// Shared-memory slot of logical FFT index i: one pad slot after every 16
// entries, so the stride-8 writes of the first Stockham stages hit distinct
// banks (without it a warp's stage-1 store of 8-byte values is 16-way conflicted).
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// Shared-memory slots of one group: the padded FFT buffer (pidx(M-1) <
// M + M/16) and four spare complex slots after it, where the line's border
// coefficients are left for every thread of the group.
__host__ __device__ __forceinline__ int group_slots(int M) { return M + M / 16 + 4; }

template <typename T> __device__ __forceinline__ void dft4(C2<T>& a0, C2<T>& a1, C2<T>& a2, C2<T>& a3) {
    const C2<T> s02 = cadd<T>(a0, a2), d02 = csub<T>(a0, a2);
    const C2<T> s13 = cadd<T>(a1, a3), d13 = csub<T>(a1, a3);
    const C2<T> md13 = cmk<T>(d13.y, -d13.x);          // -i * d13
    a0 = cadd<T>(s02, s13);
    a2 = csub<T>(s02, s13);
    a1 = cadd<T>(d02, md13);
    a3 = csub<T>(d02, md13);
}

template <typename T> __device__ __forceinline__ void dft8(C2<T>* v) {
    C2<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C2<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<T>(e0, e1, e2, e3);
    dft4<T>(o0, o1, o2, o3);
    const T c = (T)0.70710678118654752440;
    const C2<T> w1 = cmk<T>(c * (o1.x + o1.y), c * (o1.y - o1.x));     // exp(-i pi/4) o1
    const C2<T> w2 = cmk<T>(o2.y, -o2.x);                             // -i o2
    const C2<T> w3 = cmk<T>(c * (o3.y - o3.x), -c * (o3.x + o3.y));   // exp(-3i pi/4) o3
    v[0] = cadd<T>(e0, o0); v[4] = csub<T>(e0, o0);
    v[1] = cadd<T>(e1, w1); v[5] = csub<T>(e1, w1);
    v[2] = cadd<T>(e2, w2); v[6] = csub<T>(e2, w2);
    v[3] = cadd<T>(e3, w3); v[7] = csub<T>(e3, w3);
}

// One Stockham autosort stage of radix R on buf[0..M): butterfly j reads
// buf[j + r M/R], twiddles by W_{Ns R}^{r (j mod Ns)}, does an R-point DFT, and
// writes buf[(j - j mod Ns) R + j mod Ns + r Ns].  Each thread holds 8 values.
// tws is this stage's twiddle table, laid out [power][k] (powers 1, 2, 4 of
// W_{Ns R}^k, k < Ns) so a warp's loads are contiguous; the other powers are
// formed with one complex product each (two roundings at most).
// FIRST marks the stage with Ns = 1 (no twiddles); it reads positions < lim_in
// only (the rest are zero: the Bluestein padding) and, with PRE, multiplies
// each value read by pre[] and conjugates it (the chirp product between the
// two Bluestein FFTs).  Writes at positions >= lim_out are dropped (outputs
// nobody reads).
template <int R, bool FIRST, bool PRE, typename T>
__device__ __forceinline__ void fft_stage(C2<T>* buf, int M, int Ns, const C2<T>* __restrict__ tws,
                                          const C2<T>* __restrict__ pre, int lim_in, int lim_out,
                                          int t, int tpg) {
    constexpr int PER = 8 / R;
    const int nb = M / R;
    C2<T> v[8];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = t + u * tpg;
        const int k = FIRST ? 0 : (j & (Ns - 1));
        C2<T> w[8];
        if (!FIRST) {
            w[1] = tws[k];
            if (R >= 4) w[2] = tws[Ns + k];
            if (R == 8) w[4] = tws[2 * Ns + k];
            if (R >= 4) w[3] = cmul<T>(w[1], w[2]);
            if (R == 8) {
                w[5] = cmul<T>(w[1], w[4]);
                w[6] = cmul<T>(w[2], w[4]);
                w[7] = cmul<T>(w[3], w[4]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int p = j + r * nb;
            C2<T> x;
            if (FIRST) {
                x = cmk<T>(0, 0);
                if (p < lim_in) {
                    x = buf[pidx(p)];
                    if (PRE) x = cconj<T>(cmul<T>(x, pre[p]));
                }
            } else {
                x = buf[pidx(p)];
                if (r > 0) x = cmul<T>(x, w[r]);
            }
            v[u * R + r] = x;
        }
        if (R == 8) dft8<T>(v + u * R);
        else if (R == 4) dft4<T>(v[u * R], v[u * R + 1], v[u * R + 2], v[u * R + 3]);
        else {
            const C2<T> a = v[u * R], b = v[u * R + 1];
            v[u * R] = cadd<T>(a, b);
            v[u * R + 1] = csub<T>(a, b);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = t + u * tpg;
        const int k = FIRST ? 0 : (j & (Ns - 1));
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (base + r * Ns < lim_out) buf[pidx(base + r * Ns)] = v[u * R + r];
    }
    __syncthreads();
}

// The same stage with the sub-length NS fixed at compile time, for M >= 128
// (so nb = M/R and tpg = M/8 are multiples of 16).  Shared-memory slots then
// follow from one pidx per butterfly: pidx(j + r nb) = pidx(j) + r (nb + nb/16)
// because nb is a multiple of 16, and pidx(base + r NS) = pidx(base) + pidx(r NS)
// because the low four bits of base and r NS never carry (NS = 1: base = 8j;
// NS = 8: base mod 16 = j mod 8; NS >= 64: r NS mod 16 = 0).  IN: 0 plain
// reads, 1 reads at positions >= lim_in taken as zero, 2 the pre[] product;
// OUTLIM: writes at positions >= lim_out dropped.
template <int R, int NS, int IN, bool OUTLIM, typename T>
__device__ __forceinline__ void fft_stage_ct(C2<T>* buf, int nb, const C2<T>* __restrict__ tws,
                                             const C2<T>* __restrict__ pre, int lim_in, int lim_out, int t,
                                             int tpg) {
    constexpr int PER = 8 / R;
    const int rstep = nb + (nb >> 4);
    const int pt = pidx(t), tstep = tpg + (tpg >> 4);
    C2<T> v[8];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = t + u * tpg;
        const int pj = pt + u * tstep;
        const int k = j & (NS - 1);
        C2<T> w[8];
        if (NS > 1) {
            w[1] = tws[k];
            if (R >= 4) w[2] = tws[NS + k];
            if (R == 8) w[4] = tws[2 * NS + k];
            if (R >= 4) w[3] = cmul<T>(w[1], w[2]);
            if (R == 8) {
                w[5] = cmul<T>(w[1], w[4]);
                w[6] = cmul<T>(w[2], w[4]);
                w[7] = cmul<T>(w[3], w[4]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C2<T> x;
            if (IN == 1) {
                x = cmk<T>(0, 0);
                if (j + r * nb < lim_in) x = buf[pj + r * rstep];
            } else {
                x = buf[pj + r * rstep];
                if (IN == 2) x = cconj<T>(cmul<T>(x, pre[j + r * nb]));
            }
            if (NS > 1 && r > 0) x = cmul<T>(x, w[r]);
            v[u * R + r] = x;
        }
        if (R == 8) dft8<T>(v + u * R);
        else if (R == 4) dft4<T>(v[u * R], v[u * R + 1], v[u * R + 2], v[u * R + 3]);
        else {
            const C2<T> a = v[u * R], b = v[u * R + 1];
            v[u * R] = cadd<T>(a, b);
            v[u * R + 1] = csub<T>(a, b);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = t + u * tpg;
        const int k = j & (NS - 1);
        const int base = (j - k) * R + k;
        const int pb = pidx(base);
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (!OUTLIM || base + r * NS < lim_out) buf[pb + r * NS + ((r * NS) >> 4)] = v[u * R + r];
    }
    __syncthreads();
}

// Stages of 128 <= M <= 4096 with every sub-length fixed at compile time:
// radix 8 at NS = 1 and 8, then radix 8, 4 or 2 at NS = 64 and, for M >= 1024,
// at NS = 512 (twiddle tables at offsets 0, 24 and 216, as the host lays them out).
template <int IN, bool OUTLIM, typename T>
__device__ __forceinline__ void group_fft_ct(C2<T>* buf, const Axis<T>& ax, int t, const C2<T>* pre, int lim_in,
                                             int lim_out) {
    const int M = ax.M, L2 = ax.log2M, tpg = ax.tpg;
    fft_stage_ct<8, 1, IN, false, T>(buf, M / 8, nullptr, pre, lim_in, lim_out, t, tpg);
    fft_stage_ct<8, 8, 0, false, T>(buf, M / 8, ax.tw, nullptr, M, M, t, tpg);
    const C2<T>* tw64 = ax.tw + 24;
    if (L2 == 7) fft_stage_ct<2, 64, 0, OUTLIM, T>(buf, M / 2, tw64, nullptr, M, lim_out, t, tpg);
    else if (L2 == 8) fft_stage_ct<4, 64, 0, OUTLIM, T>(buf, M / 4, tw64, nullptr, M, lim_out, t, tpg);
    else if (L2 == 9) fft_stage_ct<8, 64, 0, OUTLIM, T>(buf, M / 8, tw64, nullptr, M, lim_out, t, tpg);
    else {
        fft_stage_ct<8, 64, 0, false, T>(buf, M / 8, tw64, nullptr, M, M, t, tpg);
        const C2<T>* tw512 = ax.tw + 216;
        if (L2 == 10) fft_stage_ct<2, 512, 0, OUTLIM, T>(buf, M / 2, tw512, nullptr, M, lim_out, t, tpg);
        else if (L2 == 11) fft_stage_ct<4, 512, 0, OUTLIM, T>(buf, M / 4, tw512, nullptr, M, lim_out, t, tpg);
        else fft_stage_ct<8, 512, 0, OUTLIM, T>(buf, M / 8, tw512, nullptr, M, lim_out, t, tpg);
    }
}

// 16-point DFT in registers, split as r = r1 + 4 r2 and k = s + 4 k1:
// X_{s + 4 k1} = sum_{r1} W4^{r1 k1} [W16^{r1 s} sum_{r2} W4^{r2 s} x_{r1 + 4 r2}]:
// four DFT4s over r2, the nine non-trivial W16 factors, four DFT4s over r1.
template <typename T> __device__ __forceinline__ void dft16(C2<T>* v) {
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) dft4<T>(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]);
    const T c1 = (T)0.92387953251128675613;     // cos(pi/8)
    const T s1 = (T)0.38268343236508977173;     // sin(pi/8)
    const T c2 = (T)0.70710678118654752440;     // cos(pi/4)
    // y[r1][s] sits in v[r1 + 4 s]; multiply by W16^{r1 s} = exp(-2 pi i r1 s / 16)
    v[5] = cmul<T>(v[5], cmk<T>(c1, -s1));                          // W^1
    v[9] = cmk<T>(c2 * (v[9].x + v[9].y), c2 * (v[9].y - v[9].x));  // W^2
    v[13] = cmul<T>(v[13], cmk<T>(s1, -c1));                        // W^3
    v[6] = cmk<T>(c2 * (v[6].x + v[6].y), c2 * (v[6].y - v[6].x));  // W^2
    v[10] = cmk<T>(v[10].y, -v[10].x);                              // W^4 = -i
    v[14] = cmk<T>(c2 * (v[14].y - v[14].x), -c2 * (v[14].x + v[14].y));   // W^6
    v[7] = cmul<T>(v[7], cmk<T>(s1, -c1));                          // W^3
    v[11] = cmk<T>(c2 * (v[11].y - v[11].x), -c2 * (v[11].x + v[11].y));   // W^6
    v[15] = cmul<T>(v[15], cmk<T>(-c1, s1));                        // W^9
#pragma unroll
    for (int s = 0; s < 4; ++s) dft4<T>(v[4 * s], v[4 * s + 1], v[4 * s + 2], v[4 * s + 3]);
    // X_q now sits in v[dft16_slot(q)] (q = s + 4 k1 in v[4 s + k1])
}
__host__ __device__ __forceinline__ constexpr int dft16_slot(int q) { return 4 * (q & 3) + (q >> 2); }

// FFT lengths M >= 256 run with 16 values per thread (radix-16 stages, M/16
// threads per group), smaller ones with 8 (radix-8 stages, M/8 threads).
// Default radix of an FFT of length M: radix-16 stages from M = 256 up (the
// batched path's autotuned schedule may choose radix 8 instead).
__host__ __device__ __forceinline__ bool fft_r16(int M) { return M >= 256; }

// A stage of the 16-values-per-thread FFT: PER = 16/R butterflies of radix R
// per thread, the sub-length NS fixed at compile time, slot arithmetic as in
// fft_stage_ct (nb = M/R and tpg = M/16 are multiples of 16; NS is 1, 16 or 256).
// Radix-16 twiddles W_{16 NS}^{r k}: powers 1, 2, 3, 4, 8, 12 are loaded and
// the rest formed with one complex product (W^{a + 4 b} = W^a W^{4 b}).
template <int R, int NS, int IN, bool OUTLIM, typename T>
__device__ __forceinline__ void fft_stage16(C2<T>* buf, int nb, const C2<T>* __restrict__ tws,
                                            const C2<T>* __restrict__ pre, int lim_in, int lim_out, int t,
                                            int tpg) {
    constexpr int PER = 16 / R;
    const int rstep = nb + (nb >> 4);
    const int pt = pidx(t), tstep = tpg + (tpg >> 4);
    C2<T> v[16];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = t + u * tpg;
        const int pj = pt + u * tstep;
        const int k = j & (NS - 1);
        C2<T> wl[4], wh[4], w8[8];
        if (NS > 1) {
            if (R == 16) {
                wl[1] = tws[k]; wl[2] = tws[NS + k]; wl[3] = tws[2 * NS + k];
                wh[1] = tws[3 * NS + k]; wh[2] = tws[4 * NS + k]; wh[3] = tws[5 * NS + k];
            } else {
                w8[1] = tws[k];
                if (R >= 4) w8[2] = tws[NS + k];
                if (R == 8) w8[4] = tws[2 * NS + k];
                if (R >= 4) w8[3] = cmul<T>(w8[1], w8[2]);
                if (R == 8) {
                    w8[5] = cmul<T>(w8[1], w8[4]);
                    w8[6] = cmul<T>(w8[2], w8[4]);
                    w8[7] = cmul<T>(w8[3], w8[4]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C2<T> x;
            if (IN == 1) {
                x = cmk<T>(0, 0);
                if (j + r * nb < lim_in) x = buf[pj + r * rstep];
            } else {
                x = buf[pj + r * rstep];
                if (IN == 2) x = cconj<T>(cmul<T>(x, pre[j + r * nb]));
            }
            if (NS > 1 && r > 0) {
                if (R == 16) {
                    const int lo = r & 3, hi = r >> 2;
                    const C2<T> w = lo == 0 ? wh[hi] : (hi == 0 ? wl[lo] : cmul<T>(wl[lo], wh[hi]));
                    x = cmul<T>(x, w);
                } else {
                    x = cmul<T>(x, w8[r]);
                }
            }
            v[u * R + r] = x;
        }
        if (R == 16) dft16<T>(v);
        else if (R == 8) dft8<T>(v + u * R);
        else if (R == 4) dft4<T>(v[u * R], v[u * R + 1], v[u * R + 2], v[u * R + 3]);
        else {
            const C2<T> a = v[u * R], b = v[u * R + 1];
            v[u * R] = cadd<T>(a, b);
            v[u * R + 1] = csub<T>(a, b);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = t + u * tpg;
        const int k = j & (NS - 1);
        const int base = (j - k) * R + k;
        const int pb = pidx(base);
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (!OUTLIM || base + r * NS < lim_out)
                buf[pb + r * NS + ((r * NS) >> 4)] = v[R == 16 ? dft16_slot(r) : u * R + r];
    }
    __syncthreads();
}

// Stages of 256 <= M <= 4096: radix 16 at NS = 1 and 16, then radix 2, 4, 8
// or 16 at NS = 256 for M >= 512 (twiddle tables at offsets 0 and 96).
template <int IN, bool OUTLIM, typename T>
__device__ __forceinline__ void group_fft16(C2<T>* buf, const Axis<T>& ax, int t, const C2<T>* pre, int lim_in,
                                            int lim_out) {
    const int M = ax.M, L2 = ax.log2M, tpg = ax.tpg;
    fft_stage16<16, 1, IN, false, T>(buf, M / 16, nullptr, pre, lim_in, lim_out, t, tpg);
    if (L2 == 8) {
        fft_stage16<16, 16, 0, OUTLIM, T>(buf, M / 16, ax.tw, nullptr, M, lim_out, t, tpg);
        return;
    }
    fft_stage16<16, 16, 0, false, T>(buf, M / 16, ax.tw, nullptr, M, M, t, tpg);
    const C2<T>* tw256 = ax.tw + 96;
    if (L2 == 9) fft_stage16<2, 256, 0, OUTLIM, T>(buf, M / 2, tw256, nullptr, M, lim_out, t, tpg);
    else if (L2 == 10) fft_stage16<4, 256, 0, OUTLIM, T>(buf, M / 4, tw256, nullptr, M, lim_out, t, tpg);
    else if (L2 == 11) fft_stage16<8, 256, 0, OUTLIM, T>(buf, M / 8, tw256, nullptr, M, lim_out, t, tpg);
    else fft_stage16<16, 256, 0, OUTLIM, T>(buf, M / 16, tw256, nullptr, M, lim_out, t, tpg);
}

// Forward power-of-two FFT (exp(-i ...)) of buf[0..M) in place.  Every thread of
// the CTA must call it (it synchronises the CTA); t in [0, M/8).  The first
// stage (radix 8: M >= 8) reads positions < lim_in (the rest are zero) and,
// with PRE, applies the pre[] product; the last stage writes positions < lim_out only.
template <bool PRE, typename T>
__device__ __forceinline__ void group_fft(C2<T>* buf, const Axis<T>& ax, int t, const C2<T>* pre, int lim_in,
                                          int lim_out) {
    const int M = ax.M;
    int rem = ax.log2M - 3;
    fft_stage<8, true, PRE, T>(buf, M, 1, nullptr, pre, lim_in, rem == 0 ? lim_out : M, t, ax.tpg);
    int Ns = 8, off = 0;
    while (rem >= 3) {
        rem -= 3;
        fft_stage<8, false, false, T>(buf, M, Ns, ax.tw + off, nullptr, M, rem == 0 ? lim_out : M, t, ax.tpg);
        off += 3 * Ns;
        Ns <<= 3;
    }
    if (rem == 2) fft_stage<4, false, false, T>(buf, M, Ns, ax.tw + off, nullptr, M, lim_out, t, ax.tpg);
    else if (rem == 1) fft_stage<2, false, false, T>(buf, M, Ns, ax.tw + off, nullptr, M, lim_out, t, ax.tpg);
}

// Input side of the length-L DFT: value placed at position p of the core.
template <typename T>
__device__ __forceinline__ C2<T> dft_in(const Axis<T>& ax, int p, C2<T> x) {
    return ax.blue ? cmul<T>(x, ax.chirp[p]) : x;
}

// The length-L DFT of what dft_in placed in buf[0..L) (nothing needs to be
// stored at positions >= L: the first stage reads them as zero).  Leaves buf
// such that dft_out(k), k < L, is output k; positions >= L are left undefined.
template <typename T>
__device__ __forceinline__ void group_dft(C2<T>* buf, const Axis<T>& ax, int t) {
    const bool r16 = ax.r16;
    const bool ct = ax.log2M >= 7 && ax.log2M <= 12;
    if (ax.blue) {
        // the second FFT's first stage applies the pointwise product with the
        // transformed chirp, conjugated so the second forward FFT computes the
        // inverse (1/M folded into bhat); only outputs k < L are kept
        if (r16) {
            group_fft16<1, false, T>(buf, ax, t, nullptr, ax.L, ax.M);
            group_fft16<2, true, T>(buf, ax, t, ax.bhat, ax.M, ax.L);
        } else if (ct) {
            group_fft_ct<1, false, T>(buf, ax, t, nullptr, ax.L, ax.M);
            group_fft_ct<2, true, T>(buf, ax, t, ax.bhat, ax.M, ax.L);
        } else {
            group_fft<false, T>(buf, ax, t, nullptr, ax.L, ax.M);
            group_fft<true, T>(buf, ax, t, ax.bhat, ax.M, ax.L);
        }
    } else if (r16) {
        group_fft16<0, false, T>(buf, ax, t, nullptr, ax.M, ax.M);
    } else if (ct) {
        group_fft_ct<0, false, T>(buf, ax, t, nullptr, ax.M, ax.M);
    } else {
        group_fft<false, T>(buf, ax, t, nullptr, ax.M, ax.M);
    }
}

template <typename T>
__device__ __forceinline__ C2<T> dft_out(const C2<T>* buf, const Axis<T>& ax, int k) {
    const C2<T> z = buf[pidx(k)];
    return ax.blue ? cmul<T>(cconj<T>(z), ax.chirp[k]) : z;
}

// Position of interior sample j in the permuted sequence whose DFT gives the
// DCT-II (even samples forward, odd samples backward).
__device__ __forceinline__ int pos_C(int j, int N) { return (j & 1) ? (N - 1 - (j >> 1)) : (j >> 1); }

// ------------------------------------------------------------- boundary

// Border coefficients (c_1, c_n) of a line y = T_X c.  Writing T_X with the
// interior block extended by continuity (Sec. 3, remark) gives, per family,
//   S: y_1 = p_1 c_1, y_n = p_1 c_n;
//   C: (q_1 - q_2) c_1 - q_{n-1} c_n = y_1 - y_2,  -q_{n-1} c_1 + (q_1 - q_2) c_n = y_n - y_{n-1};
//   F: (q_1 - q_{n-1}) c_1 - q_2 c_n = y_1 - y_{n-1},  -q_2 c_1 + (q_1 - q_{n-1}) c_n = y_n - y_2;
// a symmetric 2x2 system whose inverse [[ka, kb], [kb, ka]] is precomputed in
// double.  This is the closed form of the Sherman-Morrison-Woodbury inverse of
// Thm. 1 (the SMW inner products reduce to unit vectors because the border
// rows repeat interior rows).
// One coefficient per call (which = 0: c_1, 1: c_n), so the threads of a
// group can share the work: the FP64 pipe of this part is narrow, and every
// warp repeating the same double operations costs more than a barrier.
template <typename T>
__device__ __forceinline__ double border_coeff(const Axis<T>& ax, double y0, double y1, double ym2, double ym1,
                                               int which) {
    if (ax.fam == FAM_S) return (which ? ym1 : y0) * ax.ka;
    double r1, r2;
    if (ax.fam == FAM_C) { r1 = y0 - y1; r2 = ym1 - ym2; }
    else { r1 = y0 - ym2; r2 = ym1 - y1; }
    return which ? ax.kb * r1 + ax.ka * r2 : ax.ka * r1 + ax.kb * r2;
}

// Families with two border columns on each side (S3: degree 3; C4, F4: degree 4):
// y = sum_b c_b B_b + E w with border columns B = (B1, B2, flip B2, flip B1).
// S3's odd extension E has rows 0 and n-1 equal to minus the first and last
// interior samples and rows 1 and n-2 zero; C4's half-sample reflection has
// rows 0, 1 equal to interior rows 1, 0 (rows 3, 2 of y) and rows n-2, n-1
// equal to rows n-3, n-4; F4's periodic wrap has rows 0, 1 equal to rows n-4,
// n-3 and rows n-2, n-1 equal to rows 2, 3.  Four row combinations of y
// therefore involve only the border coefficients (S3: rows 0+2, 1, n-2,
// n-1+n-3; C4: rows 0-3, 1-2, n-2-(n-3), n-1-(n-4); F4: rows 0-(n-4),
// 1-(n-3), (n-2)-2, (n-1)-3): a 4x4 system whose inverse is precomputed in double.
// y[0..3] are the first four samples, ym[0..3] the last four (ym[3] = y_{n-1}).
template <typename T>
__device__ __forceinline__ double border_coeff4(const Axis<T>& ax, const double* y, const double* ym, int b) {
    double r[4];
    if (ax.fam == FAM_C4) {
        r[0] = y[0] - y[3]; r[1] = y[1] - y[2]; r[2] = ym[2] - ym[1]; r[3] = ym[3] - ym[0];
    } else if (ax.fam == FAM_F4) {
        r[0] = y[0] - ym[0]; r[1] = y[1] - ym[1]; r[2] = ym[2] - y[2]; r[3] = ym[3] - y[3];
    } else {
        r[0] = y[0] + y[2]; r[1] = y[1]; r[2] = ym[2]; r[3] = ym[3] + ym[1];
    }
    return ax.k4[4 * b] * r[0] + ax.k4[4 * b + 1] * r[1] + ax.k4[4 * b + 2] * r[2] + ax.k4[4 * b + 3] * r[3];
}

// value of sum_b c_b B_b at sample a (S3, C4)
template <typename T>
__device__ __forceinline__ T border_sum4(const Axis<T>& ax, const T* c, int a) {
    const int n = ax.n;
    return c[0] * ax.q[a] + c[1] * ax.q2[a] + c[2] * ax.q2[n - 1 - a] + c[3] * ax.q[n - 1 - a];
}

// --------------------------------------------------------------- angles

// theta/pi of spectral index t (0..n-1) on an axis (Eq. (eq:jcf), (eq:Ac), (eq:Af)):
// border columns have angle 0.
template <typename T>
__device__ __forceinline__ T theta_over_pi(int fam, int n, int N, int t) {
    if (fam == FAM_R) return (T)t / (T)n;                 // reflective (Eq. (eq:refm)): no border columns
    if (fam == FAM_PH || fam == FAM_P) return (T)(2 * t) / (T)n;   // periodic (Eq. (eq:permat))
    if (t == 0 || t == n - 1) return (T)0;
    if (fam == FAM_F4) return (t == 1 || t == n - 2) ? (T)0 : (T)(2 * (t - 2)) / (T)N;   // reading R17
    if (fam == FAM_S3) return (t == 1 || t == n - 2) ? (T)0 : (T)(t - 1) / (T)(N + 1);
    if (fam == FAM_C4) return (t == 1 || t == n - 2) ? (T)0 : (T)(t - 2) / (T)N;
    if (fam == FAM_S) return (T)t / (T)(N + 1);
    if (fam == FAM_C) return (T)(t - 1) / (T)N;
    return (T)(2 * (t - 1)) / (T)N;
}

// Spectral index t of stored entry c on an axis (a Fourier family stores a half
// on its last axis: the left border entries, H frequencies, the right border
// entries; elsewhere W = n and t = c).
__device__ __forceinline__ int stored_to_t(int fam, int n, int W, int c) {
    const int nb = fam_nb(fam);
    return (fam_fourier(fam) && c >= W - nb) ? n - (W - c) : c;
}

// Laplacian eigenvalue s = 2 - 2 cos(theta) = 4 sin^2(theta/2) (Sec. 4), in the
// form without cancellation near theta = 0.
__device__ __forceinline__ float sinpi_t(float x) { return sinpif(x); }
__device__ __forceinline__ double sinpi_t(double x) { return sinpi(x); }
template <typename T> __device__ __forceinline__ T lap_eig(T frac) {
    const T sp = sinpi_t(frac * (T)0.5);
    return (T)4 * sp * sp;
}

}  // namespace hobc
