// Kernels of the hot path (Donatelli, arXiv:0906.2704), templated on the
// working precision T (float / double) and the transform family:
//   k_pair_analysis   T_X^{-1} on pairs of real lines (row passes; real column passes)
//   k_pair_synthesis  T_X on pairs of real-valued lines, optional fused filter
//   k_cplx_analysis   T_F^{-1} on complex lines (column pass of the Fourier family)
//   k_cplx_synthesis  T_F on complex lines, optional fused filter
//   k_eig             eigenvalues d = z(-theta) on the spectrum layout (FP64 sums)
//   k_gcv_partials    per-CTA partial GCV sums for every mu of the grid
//   k_gcv_finalize    G(mu_j) = num/den^2 and the grid argmin, per problem
// Index conventions are those of include/hobc.h (spectrum layout).
#pragma once

#include "hobc_device.cuh"

// Register cap of the FP32 line kernels.  64 keeps eight 128-thread FFT
// groups (four 256-thread CTAs) resident per SM at the cost of a few spilled
// bytes; 72 (no spills, six groups) ran the 1024^2 passes 11% slower.  FP64
// kernels may use 128 (512 threads x 128 = the register file).
#ifndef HOBC_LINE_REGS
#define HOBC_LINE_REGS 64
#endif
#define HOBC_LINE_BOUNDS __maxnreg__(sizeof(T) == 4 ? HOBC_LINE_REGS : 128)

namespace hobc {

template <typename T, bool CPLX> struct ElemT { typedef T t; };
template <typename T> struct ElemT<T, true> { typedef C2<T> t; };

__device__ __forceinline__ float re_of(float v) { return v; }
__device__ __forceinline__ double re_of(double v) { return v; }
__device__ __forceinline__ float re_of(float2 v) { return v.x; }
__device__ __forceinline__ double re_of(double2 v) { return v.x; }
__device__ __forceinline__ float abs2_of(float v) { return v * v; }
__device__ __forceinline__ double abs2_of(double v) { return v * v; }
__device__ __forceinline__ float abs2_of(float2 v) { return v.x * v.x + v.y * v.y; }
__device__ __forceinline__ double abs2_of(double2 v) { return v.x * v.x + v.y * v.y; }

// Filter factor Phi_i D_i^{-1} = conj(d_i) / (|d_i|^2 + mu |s_i|^2) (Eq. (eq:freg)) applied to v.
__device__ __forceinline__ float apply_filter(float v, float d, float s2, float mu) {
    return v * d / (d * d + mu * s2);
}
__device__ __forceinline__ double apply_filter(double v, double d, double s2, double mu) {
    return v * d / (d * d + mu * s2);
}
__device__ __forceinline__ float2 apply_filter(float2 v, float2 d, float s2, float mu) {
    const float den = d.x * d.x + d.y * d.y + mu * s2;
    return make_float2((v.x * d.x + v.y * d.y) / den, (v.y * d.x - v.x * d.y) / den);
}
__device__ __forceinline__ double2 apply_filter(double2 v, double2 d, double s2, double mu) {
    const double den = d.x * d.x + d.y * d.y + mu * s2;
    return make_double2((v.x * d.x + v.y * d.y) / den, (v.y * d.x - v.x * d.y) / den);
}

// Where the eigenvalues, mu* and smoothing of a filtered element come from.
struct FilterDesc {
    const void* D;          // eigenvalues in the spectrum layout
    long long d_psf_stride; // elements between consecutive PSFs' eigenvalues
    int psf_per;            // 1: one PSF per problem, 0: shared
    const int* mu_idx;      // [problems] grid index of mu*
    const double* mu;       // [K] grid
    int K;                  // grid size (caller indices are clamped to [0, K))
    int lap;                // 1: Laplacian smoothing, 0: identity
    int o_fam, o_n, o_N, o_W;   // 2D: the other axis (axis 1, indexed by line)
    const double* mu_val;   // [problems] mu* itself; when set it replaces mu_idx / mu
};

// mu* of a problem; an index outside the grid is clamped so it cannot read past it.
__device__ __forceinline__ double mu_of(const FilterDesc& f, int problem) {
    if (f.mu_val) return f.mu_val[problem];
    const int k = f.mu_idx[problem];
    return f.mu[k < 0 ? 0 : (k >= f.K ? f.K - 1 : k)];
}

// 1D (mode 1): problem = line, D offset = psf(line) * stride + pos, s = s(pos).
// 2D (mode 2): problem = item, D offset = psf(item) * stride + line*lrs + pos*lcs,
//              s = s0(pos) + s1(line)  (Kronecker-sum Laplacian).
template <typename T>
__device__ __forceinline__ T smoothing2(const FilterDesc& f, int mode, const Axis<T>& ax, int line, int pos) {
    if (!f.lap) return (T)1;
    const int t = stored_to_t(ax.fam, ax.n, ax.W, pos);
    T s = lap_eig<T>(theta_over_pi<T>(ax.fam, ax.n, ax.N, t));
    if (mode == 2) {
        const int t1 = stored_to_t(f.o_fam, f.o_n, f.o_W, line);
        s += lap_eig<T>(theta_over_pi<T>(f.o_fam, f.o_n, f.o_N, t1));
    }
    return s * s;
}

// =====================================================================
// Analysis T_X^{-1} on pairs of real lines.
// Line r of item i, sample j: in[i*in_item + r*in_rs + j].
// Output spectral entry c of line r: out[i*out_item + r*out_rs + c*out_cs]
// (out_rs == 1 means a transposed store, staged so it stays coalesced).
// grid = (ceil(nlines / 2G), items), block = G * ax.tpg.
// =====================================================================
// Stage row rr (0 <= rr < 2G) of a pair kernel: row rr & 1 of group rr >> 1,
// inside that group's buffer from slot ax.sslot on (ax.sslot >= 0: above every
// slot its FFT input or output occupies), or after all groups' buffers.
template <typename E, typename T>
__device__ __forceinline__ E* stage_row(unsigned char* smem_raw, const Axis<T>& ax, int G, int rr) {
    C2<T>* base = reinterpret_cast<C2<T>*>(smem_raw);
    if (ax.sslot >= 0) return reinterpret_cast<E*>(base + (size_t)(rr >> 1) * ax.Mp + ax.sslot) + (rr & 1) * ax.W;
    return reinterpret_cast<E*>(base + (size_t)G * ax.Mp) + (size_t)rr * ax.W;
}

template <typename T, int FAM>
__device__ __forceinline__ void pair_analysis_body(const T* __restrict__ in, long long in_item, long long in_rs,
                                                   typename ElemT<T, fam_fourier(FAM)>::t* __restrict__ out,
                                                   long long out_item, long long out_rs, long long out_cs,
                                                   int nlines, const Axis<T>& ax, long long item, int r0,
                                                   unsigned char* smem_raw) {
    constexpr bool FOUR = fam_fourier(FAM);
    typedef typename ElemT<T, FOUR>::t E;
    const int G = blockDim.x / ax.tpg;
    const int g = threadIdx.x / ax.tpg;
    const int t = threadIdx.x - g * ax.tpg;
    C2<T>* buf = reinterpret_cast<C2<T>*>(smem_raw) + (size_t)g * ax.Mp;
    const int n = ax.n, N = ax.N, W = ax.W;
    const int ra = r0 + 2 * g, rb = ra + 1;
    const bool va = ra < nlines, vb = rb < nlines;
    const T* ya = in + item * in_item + (long long)(va ? ra : 0) * in_rs;
    const T* yb = in + item * in_item + (long long)(vb ? rb : 0) * in_rs;

    constexpr bool CUBIC = (FAM == FAM_S3);
    constexpr int NB = fam_nb(FAM);              // border entries on each side
    constexpr bool K2 = NB == 2;                 // two border columns on each side (S3, C4, F4)
    constexpr bool DCT = (FAM == FAM_C || FAM == FAM_C4);
    // border coefficients of both lines, one per thread: (c_1, c_n) of line a
    // then of line b, or the four coefficients of each (S3, C4, F4); none for P
    T* xs = reinterpret_cast<T*>(buf + ax.M + ax.M / 16);
    for (int l = t; l < 4 * NB; l += ax.tpg) {
        const int side = K2 ? l >> 2 : l >> 1;
        const T* y = side ? yb : ya;
        double c = 0;
        if (side ? vb : va) {
            if constexpr (K2) {
                const double y4[4] = {y[0], y[1], y[2], y[3]};
                const double ym4[4] = {y[n - 4], y[n - 3], y[n - 2], y[n - 1]};
                c = border_coeff4<T>(ax, y4, ym4, l & 3);
            } else {
                c = border_coeff<T>(ax, y[0], y[1], y[n - 2], y[n - 1], l & 1);
            }
        }
        xs[l] = (T)c;
    }
    __syncthreads();
    T c1af = 0, cnaf = 0, c1bf = 0, cnbf = 0;
    if constexpr (NB == 1) { c1af = xs[0]; cnaf = xs[1]; c1bf = xs[2]; cnbf = xs[3]; }
    T ca4f[4] = {0, 0, 0, 0}, cb4f[4] = {0, 0, 0, 0};
    if constexpr (K2)
#pragma unroll
        for (int b = 0; b < 4; ++b) { ca4f[b] = xs[b]; cb4f[b] = xs[4 + b]; }
    const C2<T> zero = cmk<T>(0, 0);

    for (int j = t; j < N; j += ax.tpg) {
        T wa, wb;
        if constexpr (K2) {
            wa = va ? ya[2 + j] - border_sum4<T>(ax, ca4f, 2 + j) : (T)0;
            wb = vb ? yb[2 + j] - border_sum4<T>(ax, cb4f, 2 + j) : (T)0;
        } else if constexpr (NB == 0) {
            wa = va ? ya[j] : (T)0;
            wb = vb ? yb[j] : (T)0;
        } else {
            const T ql = ax.q[1 + j], qr = ax.q[n - 2 - j];
            wa = va ? ya[1 + j] - ql * c1af - qr * cnaf : (T)0;
            wb = vb ? yb[1 + j] - ql * c1bf - qr * cnbf : (T)0;
        }
        if constexpr (FOUR) {
            buf[pidx(j)] = dft_in<T>(ax, j, cmk<T>(wa, wb));
        } else if constexpr (DCT) {
            const int p = pos_C(j, N);
            buf[pidx(p)] = dft_in<T>(ax, p, cmk<T>(wa, wb));
        } else {   // odd extension of length 2(N+1)
            buf[pidx(1 + j)] = dft_in<T>(ax, 1 + j, cmk<T>(wa, wb));
            const int p2 = ax.L - 1 - j;
            buf[pidx(p2)] = dft_in<T>(ax, p2, cmk<T>(-wa, -wb));
        }
    }
    if ((FAM == FAM_S || CUBIC) && t == 0) { buf[pidx(0)] = zero; buf[pidx(N + 1)] = zero; }
    __syncthreads();
    group_dft<T>(buf, ax, t);

    E* sa = stage_row<E, T>(smem_raw, ax, G, 2 * g);
    E* sb = stage_row<E, T>(smem_raw, ax, G, 2 * g + 1);
    if constexpr (FOUR) {
        for (int k = t; k < ax.H; k += ax.tpg) {
            const C2<T> zk = dft_out<T>(buf, ax, k);
            const C2<T> zr = cconj<T>(dft_out<T>(buf, ax, k == 0 ? 0 : N - k));
            const C2<T> s = cadd<T>(zk, zr), d = csub<T>(zk, zr);
            const T h = (T)0.5 * ax.sc;
            sa[NB + k] = cmk<T>(s.x * h, s.y * h);
            sb[NB + k] = cmk<T>(d.y * h, -d.x * h);       // -i (zk - zr) / 2
        }
        if (t == 0) {
            if constexpr (K2) {
                sa[0] = cmk<T>(xs[0], 0); sa[1] = cmk<T>(xs[1], 0); sa[W - 2] = cmk<T>(xs[2], 0);
                sa[W - 1] = cmk<T>(xs[3], 0);
                sb[0] = cmk<T>(xs[4], 0); sb[1] = cmk<T>(xs[5], 0); sb[W - 2] = cmk<T>(xs[6], 0);
                sb[W - 1] = cmk<T>(xs[7], 0);
            } else if constexpr (NB == 1) {
                sa[0] = cmk<T>(xs[0], 0); sa[W - 1] = cmk<T>(xs[1], 0);
                sb[0] = cmk<T>(xs[2], 0); sb[W - 1] = cmk<T>(xs[3], 0);
            }
        }
    } else if constexpr (DCT) {
        for (int k = t; k < N; k += ax.tpg) {
            const C2<T> v = dft_out<T>(buf, ax, k);
            const C2<T> vr = cconj<T>(dft_out<T>(buf, ax, k == 0 ? 0 : N - k));
            const C2<T> s = cadd<T>(v, vr), d = csub<T>(v, vr);
            // Va = s/2, Vb = -i d/2; DCT-II coefficient = scale * Re(post_k * V)
            const C2<T> ph = ax.post[k];
            const T sk = (k == 0 ? ax.s0 : ax.s1) * (T)0.5;
            sa[NB + k] = (T)(sk * (ph.x * s.x - ph.y * s.y));
            sb[NB + k] = (T)(sk * (ph.x * d.y + ph.y * d.x));
        }
        if (t == 0) {
            if constexpr (K2) {
                sa[0] = xs[0]; sa[1] = xs[1]; sa[W - 2] = xs[2]; sa[W - 1] = xs[3];
                sb[0] = xs[4]; sb[1] = xs[5]; sb[W - 2] = xs[6]; sb[W - 1] = xs[7];
            } else {
                sa[0] = xs[0]; sa[W - 1] = xs[1]; sb[0] = xs[2]; sb[W - 1] = xs[3];
            }
        }
    } else {
        for (int k = t; k < N; k += ax.tpg) {
            const C2<T> z = dft_out<T>(buf, ax, k + 1);
            sa[NB + k] = (T)(-z.y * ax.sc);
            sb[NB + k] = (T)(z.x * ax.sc);
        }
        if (t == 0) {
            if constexpr (CUBIC) {
                sa[0] = xs[0]; sa[1] = xs[1]; sa[W - 2] = xs[2]; sa[W - 1] = xs[3];
                sb[0] = xs[4]; sb[1] = xs[5]; sb[W - 2] = xs[6]; sb[W - 1] = xs[7];
            } else {
                sa[0] = xs[0]; sa[W - 1] = xs[1]; sb[0] = xs[2]; sb[W - 1] = xs[3];
            }
        }
    }
    __syncthreads();

    const int rows_here = min(2 * G, nlines - r0);
    E* o = out + item * out_item + (long long)r0 * out_rs;
    const int total = rows_here * W;
    if (out_rs == 1) {
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int c = idx / rows_here, rr = idx - c * rows_here;
            o[rr + (long long)c * out_cs] = stage_row<E, T>(smem_raw, ax, G, rr)[c];
        }
    } else {
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int rr = idx / W, c = idx - rr * W;
            o[(long long)rr * out_rs + (long long)c * out_cs] = stage_row<E, T>(smem_raw, ax, G, rr)[c];
        }
    }
}

template <typename T, int FAM>
__global__ void HOBC_LINE_BOUNDS
k_pair_analysis(const T* __restrict__ in, long long in_item, long long in_rs,
                typename ElemT<T, fam_fourier(FAM)>::t* __restrict__ out, long long out_item,
                long long out_rs, long long out_cs, int nlines, Axis<T> ax) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = blockDim.x / ax.tpg;
    pair_analysis_body<T, FAM>(in, in_item, in_rs, out, out_item, out_rs, out_cs, nlines, ax, blockIdx.y,
                               blockIdx.x * 2 * G, smem_raw);
}

// =====================================================================
// Synthesis T_X on pairs of lines whose result is real.
// Input spectral entry c of line r: in[i*in_item + r*in_rs + c*in_cs];
// output sample j of line r: out[i*out_item + r*out_rs + j].
// FMODE 0: plain; 1: 1D filter (problem = line); 2: 2D filter (problem = item,
// the line index is the axis-1 stored index).
// =====================================================================
template <typename T, int FAM, int FMODE>
__device__ __forceinline__ void pair_synthesis_body(const typename ElemT<T, fam_fourier(FAM)>::t* __restrict__ in,
                                                    long long in_item, long long in_rs, long long in_cs,
                                                    T* __restrict__ out, long long out_item, long long out_rs,
                                                    int nlines, const Axis<T>& ax, const FilterDesc& fd,
                                                    long long item, int r0, unsigned char* smem_raw) {
    constexpr bool FOUR = fam_fourier(FAM);
    constexpr int NBF = fam_nb(FAM);
    typedef typename ElemT<T, FOUR>::t E;
    const int G = blockDim.x / ax.tpg;
    const int g = threadIdx.x / ax.tpg;
    const int t = threadIdx.x - g * ax.tpg;
    C2<T>* buf = reinterpret_cast<C2<T>*>(smem_raw) + (size_t)g * ax.Mp;
    const int n = ax.n, N = ax.N, W = ax.W;
    const int rows_here = min(2 * G, nlines - r0);

    // gather (and filter) the spectra of this CTA's lines into the stage
    {
        const E* ip = in + item * in_item + (long long)r0 * in_rs;
        const int total = rows_here * W;
        const E* Dp = reinterpret_cast<const E*>(fd.D);
        T mu_item = 0;                      // 2D filter: one mu per item, read once
        if constexpr (FMODE == 2) mu_item = (T)mu_of(fd, (int)item);
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            int rr, c;
            if (in_rs == 1) { c = idx / rows_here; rr = idx - c * rows_here; }
            else { rr = idx / W; c = idx - rr * W; }
            const long long off = (long long)rr * in_rs + (long long)c * in_cs;
            E v = ip[off];
            if constexpr (FMODE == 1) {
                const int line = r0 + rr;
                const E d = Dp[(fd.psf_per ? (long long)line : 0) * fd.d_psf_stride + c];
                const T mu = (T)mu_of(fd, line);
                v = apply_filter(v, d, smoothing2<T>(fd, 1, ax, line, c), mu);
            } else if constexpr (FMODE == 2) {
                const int line = r0 + rr;
                const E d = Dp[(fd.psf_per ? item : 0) * fd.d_psf_stride + (long long)line * in_rs + (long long)c * in_cs];
                v = apply_filter(v, d, smoothing2<T>(fd, 2, ax, line, c), mu_item);
            }
            stage_row<E, T>(smem_raw, ax, G, rr)[c] = v;
        }
        for (int idx = total + threadIdx.x; idx < 2 * G * W; idx += blockDim.x)
            stage_row<E, T>(smem_raw, ax, G, idx / W)[idx % W] = E();
    }
    __syncthreads();

    const E* sa = stage_row<E, T>(smem_raw, ax, G, 2 * g);
    const E* sb = stage_row<E, T>(smem_raw, ax, G, 2 * g + 1);
    // the border coefficients, read before the FFT may overwrite the stage
    const T c1a = re_of(sa[0]), cna = re_of(sa[W - 1]);
    const T c1b = re_of(sb[0]), cnb = re_of(sb[W - 1]);
    T c4a[4], c4b[4];
    if constexpr (NBF == 2) {
        c4a[0] = re_of(sa[0]); c4a[1] = re_of(sa[1]); c4a[2] = re_of(sa[W - 2]); c4a[3] = re_of(sa[W - 1]);
        c4b[0] = re_of(sb[0]); c4b[1] = re_of(sb[1]); c4b[2] = re_of(sb[W - 2]); c4b[3] = re_of(sb[W - 1]);
    }
    const C2<T> zero = cmk<T>(0, 0);
    if constexpr (FOUR) {
        const int H = ax.H;
        for (int k = t; k < N; k += ax.tpg) {
            C2<T> z;
            if (k < H) {
                C2<T> a = reinterpret_cast<const C2<T>*>(sa)[NBF + k];
                C2<T> b = reinterpret_cast<const C2<T>*>(sb)[NBF + k];
                if (k == 0 || 2 * k == N) { a.y = 0; b.y = 0; }
                z = cmk<T>(a.x - b.y, a.y + b.x);                // a + i b
            } else {
                const C2<T> a = reinterpret_cast<const C2<T>*>(sa)[NBF + N - k];
                const C2<T> b = reinterpret_cast<const C2<T>*>(sb)[NBF + N - k];
                z = cmk<T>(a.x + b.y, -a.y + b.x);               // conj(a) + i conj(b)
            }
            buf[pidx(k)] = dft_in<T>(ax, k, cconj<T>(z));
        }
    } else if constexpr (FAM == FAM_C || FAM == FAM_C4) {
        constexpr int NB = (FAM == FAM_C4) ? 2 : 1;
        for (int k = t; k < N; k += ax.tpg) {
            const T isk = k == 0 ? ax.is0 : ax.is1;
            const T ya = re_of(sa[NB + k]) * isk, yb = re_of(sb[NB + k]) * isk;
            const T yar = k == 0 ? (T)0 : re_of(sa[NB + N - k]) * ax.is1;
            const T ybr = k == 0 ? (T)0 : re_of(sb[NB + N - k]) * ax.is1;
            const C2<T> ph = cconj<T>(ax.post[k]);                  // exp(+i pi k/(2N))
            const C2<T> v = cmul<T>(ph, cmk<T>(ya + ybr, yb - yar));
            buf[pidx(k)] = dft_in<T>(ax, k, cconj<T>(v));
        }
    } else {
        constexpr int NB = (FAM == FAM_S3) ? 2 : 1;
        for (int k = t; k < N; k += ax.tpg) {
            const T a = re_of(sa[NB + k]), b = re_of(sb[NB + k]);
            buf[pidx(1 + k)] = dft_in<T>(ax, 1 + k, cmk<T>(a, b));
            const int p2 = ax.L - 1 - k;
            buf[pidx(p2)] = dft_in<T>(ax, p2, cmk<T>(-a, -b));
        }
        if (t == 0) { buf[pidx(0)] = zero; buf[pidx(N + 1)] = zero; }
    }
    __syncthreads();
    group_dft<T>(buf, ax, t);

    const int ra = r0 + 2 * g, rb = ra + 1;
    const bool va = ra < nlines, vb = rb < nlines;
    T* oa = out + item * out_item + (long long)ra * out_rs;
    T* ob = out + item * out_item + (long long)rb * out_rs;
    // interior sample j of the trigonometric part, for both lines
    auto wval = [&](int j, T& wa, T& wb) {
        if constexpr (FOUR) {
            const C2<T> z = dft_out<T>(buf, ax, j);
            wa = z.x * ax.sc;
            wb = -z.y * ax.sc;
        } else if constexpr (FAM == FAM_C || FAM == FAM_C4) {
            const C2<T> z = dft_out<T>(buf, ax, pos_C(j, N));
            wa = z.x * ax.invN;
            wb = -z.y * ax.invN;
        } else {
            const C2<T> z = dft_out<T>(buf, ax, j + 1);
            wa = -z.y * ax.sc;
            wb = z.x * ax.sc;
        }
    };
    if constexpr (NBF == 0) {
        for (int j = t; j < N; j += ax.tpg) {
            T wa, wb;
            wval(j, wa, wb);
            if (va) oa[j] = wa;
            if (vb) ob[j] = wb;
        }
        return;
    }
    if constexpr (NBF == 2) {
        for (int j = t; j < N; j += ax.tpg) {
            T wa, wb;
            wval(j, wa, wb);
            if (va) oa[2 + j] = wa + border_sum4<T>(ax, c4a, 2 + j);
            if (vb) ob[2 + j] = wb + border_sum4<T>(ax, c4b, 2 + j);
        }
        if (FAM == FAM_F4 && t == 0) {
            // periodic wrap: rows 0, 1 add interior samples N-2, N-1 and rows
            // n-2, n-1 interior samples 0, 1
            T w0a, w0b, w1a, w1b, wNa, wNb, wMa, wMb;
            wval(0, w0a, w0b);
            wval(1, w1a, w1b);
            wval(N - 2, wMa, wMb);
            wval(N - 1, wNa, wNb);
            if (va) {
                oa[0] = border_sum4<T>(ax, c4a, 0) + wMa; oa[1] = border_sum4<T>(ax, c4a, 1) + wNa;
                oa[n - 2] = border_sum4<T>(ax, c4a, n - 2) + w0a; oa[n - 1] = border_sum4<T>(ax, c4a, n - 1) + w1a;
            }
            if (vb) {
                ob[0] = border_sum4<T>(ax, c4b, 0) + wMb; ob[1] = border_sum4<T>(ax, c4b, 1) + wNb;
                ob[n - 2] = border_sum4<T>(ax, c4b, n - 2) + w0b; ob[n - 1] = border_sum4<T>(ax, c4b, n - 1) + w1b;
            }
        } else if (FAM == FAM_C4 && t == 0) {
            // half-sample reflection: rows 0, 1 add interior samples 1, 0 and
            // rows n-2, n-1 interior samples N-1, N-2
            T w0a, w0b, w1a, w1b, wNa, wNb, wMa, wMb;
            wval(0, w0a, w0b);
            wval(1, w1a, w1b);
            wval(N - 1, wNa, wNb);
            wval(N - 2, wMa, wMb);
            if (va) {
                oa[0] = border_sum4<T>(ax, c4a, 0) + w1a; oa[1] = border_sum4<T>(ax, c4a, 1) + w0a;
                oa[n - 2] = border_sum4<T>(ax, c4a, n - 2) + wNa; oa[n - 1] = border_sum4<T>(ax, c4a, n - 1) + wMa;
            }
            if (vb) {
                ob[0] = border_sum4<T>(ax, c4b, 0) + w1b; ob[1] = border_sum4<T>(ax, c4b, 1) + w0b;
                ob[n - 2] = border_sum4<T>(ax, c4b, n - 2) + wNb; ob[n - 1] = border_sum4<T>(ax, c4b, n - 1) + wMb;
            }
        } else if (t == 0) {
            // rows 1 and n-2 carry only the border columns; rows 0 and n-1 also
            // minus the first / last interior trigonometric sample (odd extension)
            T wa0, wb0, wa1, wb1;
            wval(0, wa0, wb0);
            wval(N - 1, wa1, wb1);
            if (va) {
                oa[1] = border_sum4<T>(ax, c4a, 1); oa[n - 2] = border_sum4<T>(ax, c4a, n - 2);
                oa[0] = border_sum4<T>(ax, c4a, 0) - wa0; oa[n - 1] = border_sum4<T>(ax, c4a, n - 1) - wa1;
            }
            if (vb) {
                ob[1] = border_sum4<T>(ax, c4b, 1); ob[n - 2] = border_sum4<T>(ax, c4b, n - 2);
                ob[0] = border_sum4<T>(ax, c4b, 0) - wb0; ob[n - 1] = border_sum4<T>(ax, c4b, n - 1) - wb1;
            }
        }
        return;
    }
    for (int j = t; j < N; j += ax.tpg) {
        T wa, wb;
        wval(j, wa, wb);
        const T ql = ax.q[1 + j], qr = ax.q[n - 2 - j];
        if (va) oa[1 + j] = wa + ql * c1a + qr * cna;
        if (vb) ob[1 + j] = wb + ql * c1b + qr * cnb;
    }
    if (t == 0) {
        T wa0 = 0, wb0 = 0, wa1 = 0, wb1 = 0;
        if (FAM != FAM_S) { wval(0, wa0, wb0); wval(N - 1, wa1, wb1); }
        // C: y_1 = q_1 c_1 + w_1, y_n = q_1 c_n + w_N;  F: y_1 = q_1 c_1 + w_N, y_n = q_1 c_n + w_1
        const T fa = FAM == FAM_C ? wa0 : wa1, la = FAM == FAM_C ? wa1 : wa0;
        const T fb = FAM == FAM_C ? wb0 : wb1, lb = FAM == FAM_C ? wb1 : wb0;
        if (va) { oa[0] = ax.q1 * c1a + fa; oa[n - 1] = ax.q1 * cna + la; }
        if (vb) { ob[0] = ax.q1 * c1b + fb; ob[n - 1] = ax.q1 * cnb + lb; }
    }
}

template <typename T, int FAM, int FMODE>
__global__ void HOBC_LINE_BOUNDS
k_pair_synthesis(const typename ElemT<T, fam_fourier(FAM)>::t* __restrict__ in, long long in_item,
                 long long in_rs, long long in_cs, T* __restrict__ out, long long out_item,
                 long long out_rs, int nlines, Axis<T> ax, FilterDesc fd) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = blockDim.x / ax.tpg;
    pair_synthesis_body<T, FAM, FMODE>(in, in_item, in_rs, in_cs, out, out_item, out_rs, nlines, ax, fd,
                                       blockIdx.y, blockIdx.x * 2 * G, smem_raw);
}

// =====================================================================
// Fourier families (F, F4, P), complex lines along axis 0 (one line per thread
// group).  Line c of item i: in[i*item_stride + c*n + t].  The border solve
// of a complex line is the real one applied to its real and imaginary parts.
// =====================================================================
template <typename T, int FAM>
__global__ void HOBC_LINE_BOUNDS
k_cplx_analysis(const C2<T>* __restrict__ in, C2<T>* __restrict__ out, long long item_stride,
                int nlines, Axis<T> ax) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NB = fam_nb(FAM);
    const int G = blockDim.x / ax.tpg;
    const int g = threadIdx.x / ax.tpg;
    const int t = threadIdx.x - g * ax.tpg;
    C2<T>* buf = reinterpret_cast<C2<T>*>(smem_raw) + (size_t)g * ax.Mp;
    const int n = ax.n, N = ax.N;
    const long long item = blockIdx.y;
    const int c = blockIdx.x * G + g;
    const bool valid = c < nlines;
    const C2<T>* y = in + item * item_stride + (long long)(valid ? c : 0) * n;
    // border coefficients, one per thread: those of the real part (c_1, c_n;
    // or the four of F4), then those of the imaginary part
    T* xs = reinterpret_cast<T*>(buf + ax.M + ax.M / 16);
    for (int l = t; l < 4 * NB; l += ax.tpg) {
        double cf = 0;
        if (valid) {
            if constexpr (NB == 2) {
                const bool im = l >= 4;
                double y4[4], ym4[4];
                for (int a = 0; a < 4; ++a) {
                    const C2<T> u = y[a], v = y[n - 4 + a];
                    y4[a] = im ? u.y : u.x;
                    ym4[a] = im ? v.y : v.x;
                }
                cf = border_coeff4<T>(ax, y4, ym4, l & 3);
            } else {
                const C2<T> y0 = y[0], y1 = y[1], ym2 = y[n - 2], ym1 = y[n - 1];
                cf = l < 2 ? border_coeff<T>(ax, y0.x, y1.x, ym2.x, ym1.x, l & 1)
                           : border_coeff<T>(ax, y0.y, y1.y, ym2.y, ym1.y, l & 1);
            }
        }
        xs[l] = (T)cf;
    }
    __syncthreads();
    C2<T> c1 = cmk<T>(0, 0), cn = cmk<T>(0, 0);
    T cre[4] = {0, 0, 0, 0}, cim[4] = {0, 0, 0, 0};
    if constexpr (NB == 1) { c1 = cmk<T>(xs[0], xs[2]); cn = cmk<T>(xs[1], xs[3]); }
    if constexpr (NB == 2)
#pragma unroll
        for (int b = 0; b < 4; ++b) { cre[b] = xs[b]; cim[b] = xs[4 + b]; }
    for (int j = t; j < N; j += ax.tpg) {
        C2<T> w = cmk<T>(0, 0);
        if (valid) {
            const C2<T> v = y[NB + j];
            if constexpr (NB == 2) {
                w = cmk<T>(v.x - border_sum4<T>(ax, cre, 2 + j), v.y - border_sum4<T>(ax, cim, 2 + j));
            } else if constexpr (NB == 1) {
                const T ql = ax.q[1 + j], qr = ax.q[n - 2 - j];
                w = cmk<T>(v.x - ql * c1.x - qr * cn.x, v.y - ql * c1.y - qr * cn.y);
            } else {
                w = v;
            }
        }
        buf[pidx(j)] = dft_in<T>(ax, j, w);
    }
    __syncthreads();
    group_dft<T>(buf, ax, t);
    if (!valid) return;
    C2<T>* o = out + item * item_stride + (long long)c * n;
    for (int k = t; k < N; k += ax.tpg) o[NB + k] = cscale<T>(dft_out<T>(buf, ax, k), ax.sc);
    if (t == 0) {                                   // xs outlives the FFT
        if constexpr (NB == 1) { o[0] = cmk<T>(xs[0], xs[2]); o[n - 1] = cmk<T>(xs[1], xs[3]); }
        if constexpr (NB == 2) {
            o[0] = cmk<T>(xs[0], xs[4]); o[1] = cmk<T>(xs[1], xs[5]);
            o[n - 2] = cmk<T>(xs[2], xs[6]); o[n - 1] = cmk<T>(xs[3], xs[7]);
        }
    }
}

template <typename T, int FAM, bool FILTER>
__global__ void HOBC_LINE_BOUNDS
k_cplx_synthesis(const C2<T>* __restrict__ in, C2<T>* __restrict__ out, long long item_stride,
                 int nlines, Axis<T> ax, FilterDesc fd) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NB = fam_nb(FAM);
    const int G = blockDim.x / ax.tpg;
    const int g = threadIdx.x / ax.tpg;
    const int t = threadIdx.x - g * ax.tpg;
    C2<T>* buf = reinterpret_cast<C2<T>*>(smem_raw) + (size_t)g * ax.Mp;
    const int n = ax.n, N = ax.N;
    const long long item = blockIdx.y;
    const int c = blockIdx.x * G + g;
    const bool valid = c < nlines;
    const C2<T>* x = in + item * item_stride + (long long)(valid ? c : 0) * n;
    const C2<T>* Dp = reinterpret_cast<const C2<T>*>(fd.D) + (fd.psf_per ? item : 0) * fd.d_psf_stride +
                      (long long)(valid ? c : 0) * n;
    T mu = 0;
    if (FILTER) mu = (T)mu_of(fd, (int)item);
    auto coef = [&](int pos) -> C2<T> {
        C2<T> v = x[pos];
        if constexpr (FILTER) v = apply_filter(v, Dp[pos], smoothing2<T>(fd, 2, ax, c, pos), mu);
        return v;
    };
    for (int k = t; k < N; k += ax.tpg) {
        const C2<T> v = valid ? coef(NB + k) : cmk<T>(0, 0);
        buf[pidx(k)] = dft_in<T>(ax, k, cconj<T>(v));
    }
    __syncthreads();
    group_dft<T>(buf, ax, t);
    if (!valid) return;
    C2<T>* o = out + item * item_stride + (long long)c * n;
    auto wout = [&](int j) { return cscale<T>(cconj<T>(dft_out<T>(buf, ax, j)), ax.sc); };
    if constexpr (NB == 0) {
        for (int j = t; j < N; j += ax.tpg) o[j] = wout(j);
    } else if constexpr (NB == 1) {
        const C2<T> c1 = coef(0), cn = coef(n - 1);
        for (int j = t; j < N; j += ax.tpg) {
            const C2<T> w = wout(j);
            const T ql = ax.q[1 + j], qr = ax.q[n - 2 - j];
            o[1 + j] = cmk<T>(w.x + ql * c1.x + qr * cn.x, w.y + ql * c1.y + qr * cn.y);
        }
        if (t == 0) {
            const C2<T> w0 = wout(0), wN = wout(N - 1);
            o[0] = cmk<T>(ax.q1 * c1.x + wN.x, ax.q1 * c1.y + wN.y);      // y_1 = q_1 c_1 + w_N
            o[n - 1] = cmk<T>(ax.q1 * cn.x + w0.x, ax.q1 * cn.y + w0.y);  // y_n = q_1 c_n + w_1
        }
    } else {
        T cre[4], cim[4];
        const int bpos[4] = {0, 1, n - 2, n - 1};
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const C2<T> v = coef(bpos[b]);
            cre[b] = v.x; cim[b] = v.y;
        }
        auto put = [&](int row, C2<T> w) {
            o[row] = cmk<T>(w.x + border_sum4<T>(ax, cre, row), w.y + border_sum4<T>(ax, cim, row));
        };
        for (int j = t; j < N; j += ax.tpg) put(2 + j, wout(j));
        if (t == 0) {           // periodic wrap (reading R17): rows 0, 1, n-2, n-1
            put(0, wout(N - 2)); put(1, wout(N - 1)); put(n - 2, wout(0)); put(n - 1, wout(1));
        }
    }
}

// =====================================================================
// Eigenvalues d[c][t0] = sum_{j0,j1} h[j0][j1] E0[t0][j0] E1[c][j1] with
// E[t][j] = exp(-i (j - m) theta_t)  (Eq. (eq:symbol) at -theta, Sec. 6),
// accumulated in double (FP32 plans: the column sums in float-float, below).
// 1D problems use n0 = p0 = 1 and E0 = [[1]].
// The row stage P_k = sum_j1 h[m0 + k][j1] E1[c][j1] is combined over tap
// offsets +-k:  P_k e^{-ik th} + P_{-k} e^{ik th} = A_k cos(k th) - i B_k sin(k th),
// A_k = P_k + P_{-k}, B_k = P_k - P_{-k}, so the real part costs two products
// per k (four with the imaginary part) instead of eight.
// FP32 plans sum the column stage over k in float-float (the FP64 pipe of this
// part runs at 1/64 of the FP32 rate): A_k, B_k and the table E0f = E0 split
// into hi + lo float pairs, each product by TwoProduct (an FMA gives its
// rounding error), the running sum by TwoSum (Ogita, Rump and Oishi's compensated
// dot product): within about 2^-44 of the sum of |terms|, then rounded once to
// FP32.
// grid = (npsf, W1), block = 256.
// =====================================================================

// s + r += (xh + xl)(yh + yl), s + r a float-float running sum.  The _rn
// intrinsics keep the compiler from fusing or reordering the error terms.
__device__ __forceinline__ void ff_mac(float& s, float& r, float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);
    const float pe = __fmaf_rn(xh, yh, -p);                 // xh yh = p + pe exactly
    const float sn = __fadd_rn(s, p);                       // s + p = sn + se exactly
    const float bv = __fsub_rn(sn, s);
    const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bv)), __fsub_rn(p, bv));
    s = sn;
    r += se + pe + __fmaf_rn(xh, yl, xl * yh);
}

__device__ __forceinline__ float4 ff_split(double2 v) {
    const float rh = (float)v.x, ih = (float)v.y;
    return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

template <typename T, bool CPLX>
__global__ void k_eig(const T* __restrict__ psf, long long psf_stride, int p0, int p1,
                      const double2* __restrict__ E0, const double2* __restrict__ E1,
                      const float4* __restrict__ E0f, int n0,
                      typename ElemT<T, CPLX>::t* __restrict__ D, long long d_psf_stride) {
    __shared__ double2 P[64];
    __shared__ double2 A[32], Bk[32];
    __shared__ float4 Af[32], Bf[32];      // FP32: A_k, B_k split (Af[0]: P_0)
    const int c = blockIdx.y;
    const long long ip = blockIdx.x;
    const T* h = psf + ip * psf_stride;
    const int m0 = p0 / 2;
    for (int j0 = threadIdx.x; j0 < p0; j0 += blockDim.x) {
        double re = 0, im = 0;
        for (int j1 = 0; j1 < p1; ++j1) {
            const double hv = (double)h[j0 * p1 + j1];
            const double2 e = E1[(long long)c * p1 + j1];
            re += hv * e.x;
            im += hv * e.y;
        }
        P[j0] = make_double2(re, im);
    }
    __syncthreads();
    for (int k = 1 + threadIdx.x; k <= m0; k += blockDim.x) {
        const double2 pp = P[m0 + k], pm = P[m0 - k];
        A[k] = make_double2(pp.x + pm.x, pp.y + pm.y);
        Bk[k] = make_double2(pp.x - pm.x, pp.y - pm.y);
        if constexpr (sizeof(T) == 4) {
            Af[k] = ff_split(A[k]);
            Bf[k] = ff_split(Bk[k]);
        }
    }
    if (sizeof(T) == 4 && threadIdx.x == 0) Af[0] = ff_split(P[m0]);
    __syncthreads();
    typename ElemT<T, CPLX>::t* o = D + ip * d_psf_stride + (long long)c * n0;
    if constexpr (sizeof(T) == 4) {
        for (int t0 = threadIdx.x; t0 < n0; t0 += blockDim.x) {
            const float4 c0 = Af[0];
            float rh = c0.x, rl = c0.y, ih = c0.z, il = c0.w;
            const float4* e0 = E0f + (long long)t0 * p0 + m0;
            for (int k = 1; k <= m0; ++k) {
                const float4 e = e0[k];       // (cos k th, -sin k th), each hi + lo
                const float4 a = Af[k], b = Bf[k];
                ff_mac(rh, rl, a.x, a.y, e.x, e.y);                    // re += A.re cos
                ff_mac(rh, rl, -b.z, -b.w, e.z, e.w);                  //    - B.im (-sin)
                if constexpr (CPLX) {
                    ff_mac(ih, il, a.z, a.w, e.x, e.y);                // im += A.im cos
                    ff_mac(ih, il, b.x, b.y, e.z, e.w);                //    + B.re (-sin)
                }
            }
            if constexpr (CPLX) o[t0] = cmk<T>(rh + rl, ih + il);
            else o[t0] = rh + rl;
        }
        return;
    }
    for (int t0 = threadIdx.x; t0 < n0; t0 += blockDim.x) {
        double re = P[m0].x, im = P[m0].y;
        const double2* e0 = E0 + (long long)t0 * p0 + m0;
        for (int k = 1; k <= m0; ++k) {
            const double2 e = e0[k];          // (cos k th, -sin k th)
            const double2 a = A[k], b = Bk[k];
            re += a.x * e.x - b.y * e.y;
            if constexpr (CPLX) im += a.y * e.x + b.x * e.y;
        }
        if constexpr (CPLX) o[t0] = cmk<T>((T)re, (T)im);
        else o[t0] = (T)re;
    }
}

// =====================================================================
// GCV partial sums (Eq. (eq:gcv2), (eq:mugcv)).  For every stored spectral
// element: weight w (2 for Fourier-half entries standing for a conjugate
// pair, else 1), e = w |ghat|^2, a = |d|^2 / |s|^2 (elements with s = 0 have
// sigma = 0 and are dropped).  For each mu of the grid,
//   sigma = 1/(a + mu),  num += e sigma^2,  den += w sigma.
// Grid values are taken in pairs that share one reciprocal:
// r = 1/((a+mu1)(a+mu2)), sigma1 = (a+mu2) r, sigma2 = (a+mu1) r.
// In FP32 that needs mu >= 1e-18 and a <= 1e18 so the product stays normal.
// grid = chunks * items (item-major), block = 256; partials[item][chunk][2K].
// =====================================================================
struct GcvGeom {
    int ndim;
    int fam;
    int n0, N0;         // axis 0 (2D only): spectral positions along a line
    int n1, N1, W1;     // axis of the stored index c (1D: the only axis)
    int lap;
    long long S;        // stored elements per item
    int chunk;          // elements per CTA
    int K;
    int nz, Nz;         // 3D only: the leading axis, innermost in the volume spectrum
};                      // (entry e = (c n0 + t0) nz + tz)

template <typename T> struct Pack4;
template <> struct Pack4<float> { typedef float4 t; };
template <> struct Pack4<double> { typedef double4 t; };

__device__ __forceinline__ float pair_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double pair_rcp(double x) { return 1.0 / x; }

// largest a kept in FP32 so that (a + mu1)(a + mu2) cannot overflow
template <typename T> __device__ __forceinline__ T a_cap() { return sizeof(T) == 4 ? (T)1e18 : (T)1e150; }

// The mu loop of the GCV scan over the packed elements of one CTA.  Threads
// that share a group of grid values (tpm of them, adjacent lanes) split the
// elements and combine their sums with shuffles.

// Elements per CTA of the GCV scan.  In FP32 every thread sums its share of
// the chunk in float (blocked, see gcv_scan) and converts to double once, so a
// chunk holds at most 256 elements per thread of a grid-value group; FP64 sums
// in double.
__host__ __device__ inline int gcv_threads_per_group(int K, bool fp64) {
    const int per = fp64 ? 4 : 8;            // grid values per thread
    const int groups = (K + per - 1) / per;
    int tpm = 1;
    while (tpm * 2 <= 32 && tpm * 2 * groups <= 256) tpm *= 2;
    return tpm;
}
__host__ __device__ inline int gcv_chunk_for(long long S, int K, bool fp64) {
    const long long cap = fp64 ? 1024 : (long long)min(2048, 256 * gcv_threads_per_group(K, false));
    return (int)(S < cap ? S : cap);
}

// FP64: four grid values per thread, two reciprocal-sharing pairs.
__device__ __forceinline__ void gcv_scan(const double4* __restrict__ pk, int cnt, const double* __restrict__ muT,
                                         int K, double* __restrict__ outp) {
    const int NQ = (K + 3) / 4;
    const int tpm = gcv_threads_per_group(K, true);
    const int qpp = blockDim.x / tpm;
    const int sub = threadIdx.x % tpm;
    for (int base = 0; base < NQ; base += qpp) {
        const int j0 = 4 * (base + threadIdx.x / tpm);
        double mu[4], nd[4] = {0, 0, 0, 0}, dd[4] = {0, 0, 0, 0};
#pragma unroll
        for (int u = 0; u < 4; ++u) mu[u] = j0 + u < K ? muT[j0 + u] : 1.0;
        for (int i = sub; i < cnt; i += tpm) {
            const double4 v = pk[i];
#pragma unroll
            for (int u = 0; u < 4; u += 2) {
                const double t1 = v.x + mu[u], t2 = v.x + mu[u + 1];
                const double r = 1.0 / (t1 * t2);
                const double s1 = t2 * r, s2 = t1 * r;
                dd[u] += v.z * s1;
                dd[u + 1] += v.z * s2;
                nd[u] += v.y * s1 * s1;
                nd[u + 1] += v.y * s2 * s2;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            for (int off = tpm / 2; off > 0; off >>= 1) {
                nd[u] += __shfl_down_sync(0xffffffffu, nd[u], off, tpm);
                dd[u] += __shfl_down_sync(0xffffffffu, dd[u], off, tpm);
            }
        if (sub == 0)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j0 + u < K) { outp[j0 + u] = nd[u]; outp[K + j0 + u] = dd[u]; }
    }
}

// One packed entry v = (a, e, w) evaluated at the eight grid values of mA / mB
// (lanes as in gcv_scan below), added to the packed sums.
__device__ __forceinline__ void eval_group(const float4 v, const float2 (&mA)[2], const float2 (&mB)[2],
                                           float2 (&NA)[2], float2 (&NB)[2], float2 (&DA)[2], float2 (&DB)[2]) {
    const float2 aa = make_float2(v.x, v.x), ee = make_float2(v.y, v.y), ww = make_float2(v.z, v.z);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 A = __fadd2_rn(aa, mA[h]);
        const float2 B = __fadd2_rn(aa, mB[h]);
        const float2 P = __fmul2_rn(A, B);
        const float2 R = make_float2(pair_rcp(P.x), pair_rcp(P.y));
        const float2 SA = __fmul2_rn(B, R);
        const float2 SB = __fmul2_rn(A, R);
        DA[h] = __ffma2_rn(ww, SA, DA[h]);
        DB[h] = __ffma2_rn(ww, SB, DB[h]);
        NA[h] = __ffma2_rn(__fmul2_rn(ee, SA), SA, NA[h]);
        NB[h] = __ffma2_rn(__fmul2_rn(ee, SB), SB, NB[h]);
    }
}

// As eval_group, for the first entry of a block: sets the sums instead of adding.
__device__ __forceinline__ void eval_group_first(const float4 v, const float2 (&mA)[2], const float2 (&mB)[2],
                                                 float2 (&NA)[2], float2 (&NB)[2], float2 (&DA)[2],
                                                 float2 (&DB)[2]) {
    const float2 aa = make_float2(v.x, v.x), ee = make_float2(v.y, v.y), ww = make_float2(v.z, v.z);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 A = __fadd2_rn(aa, mA[h]);
        const float2 B = __fadd2_rn(aa, mB[h]);
        const float2 P = __fmul2_rn(A, B);
        const float2 R = make_float2(pair_rcp(P.x), pair_rcp(P.y));
        const float2 SA = __fmul2_rn(B, R);
        const float2 SB = __fmul2_rn(A, R);
        DA[h] = __fmul2_rn(ww, SA);
        DB[h] = __fmul2_rn(ww, SB);
        NA[h] = __fmul2_rn(__fmul2_rn(ee, SA), SA);
        NB[h] = __fmul2_rn(__fmul2_rn(ee, SB), SB);
    }
}

// FP32: eight grid values per thread in packed f32x2 lanes.  Lanes hold
// (mu0, mu2) / (mu1, mu3) and (mu4, mu6) / (mu5, mu7), so one packed product
// forms both shared denominators of a pair of pairs and each packed op
// advances two evaluations; one rcp.approx per two evaluations.
// Summation: a thread's terms (at most 256 elements, see gcv_chunk_for) go to
// float accumulators of at most GCV_BLOCK elements each, which are added to a
// second float accumulator; the tpm threads of a group (at most 32) are then
// combined in float by a shuffle tree and each grid value's CTA sum is
// converted to double once.  Every term is non-negative, so the relative error
// of a sum is at most (depth of its summation tree) x u: 15 + 16 + 5 = 36
// roundings, 2.2e-6, against 256 + 5 for one float accumulator.  FP64
// accumulators would cost two FP64 adds per term (FP64 runs at about 1/64 of
// the FP32 rate on this part) for no gain beyond that bound.
constexpr int GCV_BLOCK = 16;
__device__ __forceinline__ void gcv_scan(const float4* __restrict__ pk, int cnt, const float* __restrict__ muT,
                                         int K, double* __restrict__ outp) {
    const int NO = (K + 7) / 8;
    const int tpm = gcv_threads_per_group(K, false);
    const int opp = blockDim.x / tpm;
    const int sub = threadIdx.x % tpm;
    for (int base = 0; base < NO; base += opp) {
        const int j0 = 8 * (base + threadIdx.x / tpm);
        float mu[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) mu[u] = j0 + u < K ? muT[j0 + u] : 1.0f;
        const float2 mA[2] = {make_float2(mu[0], mu[2]), make_float2(mu[4], mu[6])};
        const float2 mB[2] = {make_float2(mu[1], mu[3]), make_float2(mu[5], mu[7])};
        const float2 z = make_float2(0.f, 0.f);
        float2 NA[2] = {z, z}, NB[2] = {z, z}, DA[2] = {z, z}, DB[2] = {z, z};
        for (int i0 = sub; i0 < cnt; i0 += GCV_BLOCK * tpm) {
            float2 nA[2], nB[2], dA[2], dB[2];
            if (i0 + (GCV_BLOCK - 1) * tpm < cnt) {         // a full block
                eval_group_first(pk[i0], mA, mB, nA, nB, dA, dB);
#pragma unroll
                for (int r = 1; r < GCV_BLOCK; ++r) eval_group(pk[i0 + r * tpm], mA, mB, nA, nB, dA, dB);
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) { nA[h] = z; nB[h] = z; dA[h] = z; dB[h] = z; }
                for (int i = i0; i < cnt; i += tpm) eval_group(pk[i], mA, mB, nA, nB, dA, dB);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                NA[h] = __fadd2_rn(NA[h], nA[h]);
                NB[h] = __fadd2_rn(NB[h], nB[h]);
                DA[h] = __fadd2_rn(DA[h], dA[h]);
                DB[h] = __fadd2_rn(DB[h], dB[h]);
            }
        }
        float nf[8], df[8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            nf[4 * h + 0] = NA[h].x; nf[4 * h + 2] = NA[h].y;
            nf[4 * h + 1] = NB[h].x; nf[4 * h + 3] = NB[h].y;
            df[4 * h + 0] = DA[h].x; df[4 * h + 2] = DA[h].y;
            df[4 * h + 1] = DB[h].x; df[4 * h + 3] = DB[h].y;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            for (int off = tpm / 2; off > 0; off >>= 1) {
                nf[u] += __shfl_down_sync(0xffffffffu, nf[u], off, tpm);
                df[u] += __shfl_down_sync(0xffffffffu, df[u], off, tpm);
            }
        if (sub == 0)
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (j0 + u < K) { outp[j0 + u] = (double)nf[u]; outp[K + j0 + u] = (double)df[u]; }
    }
}

// |s|^2 of stored element e (1 for L = I; the Laplacian's Kronecker sum, Eq.
// (eq:L) and reading R8, on 2 or 3 axes) and its stored index c along the last
// axis.
template <typename T>
__device__ __forceinline__ T lap_s2(const GcvGeom& geo, long long e, int& c) {
    int t0 = 0, tz = 0;
    if (geo.ndim == 2) {             // e < S <= 1024 x 1024: 32-bit division
        c = (int)((unsigned)e / (unsigned)geo.n0);
        t0 = (int)e - c * geo.n0;
    } else if (geo.ndim == 3) {      // volume spectrum: e = (c n0 + t0) nz + tz
        const long long e2 = e / geo.nz;
        tz = (int)(e - e2 * geo.nz);
        c = (int)(e2 / geo.n0);
        t0 = (int)(e2 - (long long)c * geo.n0);
    } else {
        c = (int)e;
    }
    if (!geo.lap) return (T)1;
    const int t1 = stored_to_t(geo.fam, geo.n1, geo.W1, c);
    T s = lap_eig<T>(theta_over_pi<T>(geo.fam, geo.n1, geo.N1, t1));
    if (geo.ndim >= 2) s += lap_eig<T>(theta_over_pi<T>(geo.fam, geo.n0, geo.N0, t0));
    if (geo.ndim == 3) s += lap_eig<T>(theta_over_pi<T>(geo.fam, geo.nz, geo.Nz, tz));
    return s * s;
}

// The GCV terms of stored element e of a problem: x = a = |d|^2 / s^2 (capped),
// y = w |ghat|^2, z = w, with w = 2 for a Fourier entry that stands for a
// conjugate pair; an entry with s = 0 contributes nothing.
template <typename T, bool CPLX>
__device__ __forceinline__ typename Pack4<T>::t gcv_term(const typename ElemT<T, CPLX>::t& spv,
                                                         const typename ElemT<T, CPLX>::t& dpv, const GcvGeom& geo,
                                                         long long e) {
    int c;
    const T s2 = lap_s2<T>(geo, e, c);
    T w = 1;
    if (CPLX) {
        // border entries and the frequencies 0 and N/2 stand for themselves
        const int nb = fam_nb(geo.fam), k = c - nb;
        const bool self = (c < nb || c >= geo.W1 - nb || k == 0 || 2 * k == geo.N1);
        w = self ? (T)1 : (T)2;
    }
    const T lam = abs2_of(dpv);
    const T g2 = abs2_of(spv);
    typename Pack4<T>::t v;
    if (s2 > (T)0) { v.x = min(lam / s2, a_cap<T>()); v.y = w * g2; v.z = w; }
    else { v.x = (T)1; v.y = (T)0; v.z = (T)0; }
    v.w = 0;
    return v;
}

// One CTA's share of the scan: elements [e0, e0 + chunk) of one problem whose
// spectrum starts at spec_item and eigenvalues at d_item; sums go to outp[2K].
template <typename T, bool CPLX>
__device__ __forceinline__ void gcv_partials_body(const typename ElemT<T, CPLX>::t* __restrict__ spec_item,
                                                  const typename ElemT<T, CPLX>::t* __restrict__ d_item,
                                                  const T* __restrict__ muT, const GcvGeom& geo, long long e0,
                                                  double* __restrict__ outp, unsigned char* smem_raw) {
    typedef typename Pack4<T>::t P4;
    P4* pk = reinterpret_cast<P4*>(smem_raw);
    const int cnt = (int)min((long long)geo.chunk, geo.S - e0);
    const typename ElemT<T, CPLX>::t* sp = spec_item + e0;
    const typename ElemT<T, CPLX>::t* dp = d_item + e0;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) pk[i] = gcv_term<T, CPLX>(sp[i], dp[i], geo, e0 + i);
    __syncthreads();
    gcv_scan(pk, cnt, muT, geo.K, outp);
}

template <typename T, bool CPLX>
__global__ void __launch_bounds__(256, 4)
k_gcv_partials(const typename ElemT<T, CPLX>::t* __restrict__ spec, const typename ElemT<T, CPLX>::t* __restrict__ D,
               long long d_psf_stride, int psf_per, const T* __restrict__ muT, GcvGeom geo,
               double* __restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nch = (int)((geo.S + geo.chunk - 1) / geo.chunk);
    const long long item = blockIdx.x / nch;
    const int chunk = blockIdx.x - (int)(item * nch);
    gcv_partials_body<T, CPLX>(spec + item * geo.S, D + (psf_per ? item : 0) * d_psf_stride, muT, geo,
                               (long long)chunk * geo.chunk, partials + (long long)blockIdx.x * 2LL * geo.K,
                               smem_raw);
}

// ---------------------------------------------------------------------
// GCV for many small problems (1D plans): a group of TPI adjacent threads owns
// one problem and each of its threads PER grid values (8 in FP32, 4 in FP64);
// the problem's entries pass through shared memory in tiles (32 KB per CTA), every
// thread sweeps all of them for its values, so the sums need no cross-thread
// reduction: G(mu_j) = num/den^2 and the first minimiser (NaN never wins)
// come out of the same kernel.  FP32 terms are summed per tile (at most 32
// entries) in float, the tiles in a second float accumulator, and that is
// folded into FP64 every 256 entries: at most 31 + 8 roundings per sum of
// non-negative terms.  grid = ceil(items / (256 / TPI)), block = 256.
// ---------------------------------------------------------------------
template <typename T, bool CPLX, int TPI>
__global__ void __launch_bounds__(256)
k_gcv_items(const typename ElemT<T, CPLX>::t* __restrict__ spec, const typename ElemT<T, CPLX>::t* __restrict__ D,
            long long d_psf_stride, int psf_per, const T* __restrict__ muT, GcvGeom geo, int items,
            double* __restrict__ gcv, int* __restrict__ mu_idx) {
    typedef typename Pack4<T>::t P4;
    constexpr int IPC = 256 / TPI;                       // problems per CTA
    constexpr int PER = sizeof(T) == 4 ? 8 : 4;          // grid values per thread
    constexpr int GT_RAW = 32768 / (IPC * (int)sizeof(P4));
    constexpr int GT_TILE = GT_RAW > 32 ? 32 : GT_RAW;   // entries per problem and tile
    __shared__ P4 tile[IPC][GT_TILE];
    const int slot = threadIdx.x / TPI, sub = threadIdx.x % TPI;
    const long long item0 = (long long)blockIdx.x * IPC;
    const long long item = item0 + slot;
    const int K = geo.K;
    const int j0 = sub * PER;
    T mu[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) mu[u] = j0 + u < K ? muT[j0 + u] : (T)1;
    double nd[PER], dd[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) { nd[u] = 0; dd[u] = 0; }
    // FP32: packed lanes as in the grid scan; FP64: pairs sharing one reciprocal
    float2 NA[2] = {}, NB[2] = {}, DA[2] = {}, DB[2] = {};
    float2 mA[2], mB[2];
    if constexpr (sizeof(T) == 4) {
        mA[0] = make_float2((float)mu[0], (float)mu[2]); mA[1] = make_float2((float)mu[4], (float)mu[6]);
        mB[0] = make_float2((float)mu[1], (float)mu[3]); mB[1] = make_float2((float)mu[5], (float)mu[7]);
    }
    int since_fold = 0;
    for (long long e0 = 0; e0 < geo.S; e0 += GT_TILE) {
        const int cnt = (int)min((long long)GT_TILE, geo.S - e0);
        __syncthreads();
        for (int i = threadIdx.x; i < IPC * GT_TILE; i += blockDim.x) {
            const int it = i / GT_TILE, k = i - it * GT_TILE;
            const long long itm = item0 + it;
            P4 v;
            v.x = (T)1; v.y = (T)0; v.z = (T)0; v.w = (T)0;
            if (itm < items && k < cnt)
                v = gcv_term<T, CPLX>(spec[itm * geo.S + e0 + k], D[(psf_per ? itm : 0) * d_psf_stride + e0 + k], geo,
                                      e0 + k);
            tile[it][k] = v;
        }
        __syncthreads();
        if (item < items) {
            if constexpr (sizeof(T) == 4) {
                float2 nA[2] = {}, nB[2] = {}, dA[2] = {}, dB[2] = {};
#pragma unroll 4
                for (int k = 0; k < cnt; ++k) eval_group(tile[slot][k], mA, mB, nA, nB, dA, dB);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    NA[h] = __fadd2_rn(NA[h], nA[h]);
                    NB[h] = __fadd2_rn(NB[h], nB[h]);
                    DA[h] = __fadd2_rn(DA[h], dA[h]);
                    DB[h] = __fadd2_rn(DB[h], dB[h]);
                }
                since_fold += cnt;
                if (since_fold >= 256 || e0 + GT_TILE >= geo.S) {        // fold into FP64
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        nd[4 * h + 0] += NA[h].x; nd[4 * h + 2] += NA[h].y;
                        nd[4 * h + 1] += NB[h].x; nd[4 * h + 3] += NB[h].y;
                        dd[4 * h + 0] += DA[h].x; dd[4 * h + 2] += DA[h].y;
                        dd[4 * h + 1] += DB[h].x; dd[4 * h + 3] += DB[h].y;
                        NA[h] = make_float2(0.f, 0.f); NB[h] = NA[h]; DA[h] = NA[h]; DB[h] = NA[h];
                    }
                    since_fold = 0;
                }
            } else {
                for (int k = 0; k < cnt; ++k) {
                    const P4 v = tile[slot][k];
#pragma unroll
                    for (int u = 0; u < PER; u += 2) {
                        const double t1 = v.x + mu[u], t2 = v.x + mu[u + 1];
                        const double r = 1.0 / (t1 * t2);
                        const double s1 = t2 * r, s2 = t1 * r;
                        dd[u] += v.z * s1;
                        dd[u + 1] += v.z * s2;
                        nd[u] += v.y * s1 * s1;
                        nd[u + 1] += v.y * s2 * s2;
                    }
                }
            }
        }
    }
    // G at this thread's grid values, then the first minimiser across the problem's threads
    double best = INFINITY;
    int bi = 0x7fffffff;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = j0 + u;
        if (item < items && j < K) {
            const double Gv = nd[u] / (dd[u] * dd[u]);
            if (gcv) gcv[item * K + j] = Gv;
            const double key = isnan(Gv) ? INFINITY : Gv;
            if (key < best) { best = key; bi = j; }
        }
    }
#pragma unroll
    for (int off = TPI / 2; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off, TPI);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off, TPI);
        if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (sub == 0 && item < items) mu_idx[item] = bi == 0x7fffffff ? 0 : bi;
}

// Sum over the chunks of one problem of the per-CTA partial sums of grid value
// j (numerator at j, denominator at K + j of each chunk's 2K block), in chunk
// order.  (Splitting it into four interleaved accumulators measured slower.)
__device__ __forceinline__ void sum_chunks(const double* __restrict__ p, int nchunks, int K, int j, double& num,
                                           double& den) {
    num = 0;
    den = 0;
    for (int c = 0; c < nchunks; ++c) {
        num += p[(long long)c * 2 * K + j];
        den += p[(long long)c * 2 * K + K + j];
    }
}

// G(mu_j) = num_j / den_j^2 and the first index of the minimum (NaN never wins).
// Launched as one thread-block cluster per problem (launch_gcv_finalize_raw).
__global__ void k_gcv_finalize(const double* __restrict__ partials, int nchunks, int K,
                               double* __restrict__ gcv, int* __restrict__ mu_idx);

}  // namespace hobc
