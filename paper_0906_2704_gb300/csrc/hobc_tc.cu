// Dense transforms on the 5th-generation tensor cores (split-BF16).
//
// Every pass of the dense mode is C[M x N] = A[M x K] . B[N x K]^T with both
// operands K-major in HBM and each operand held as a pair of bfloat16 arrays
// (hi = bf16(x), lo = bf16(x - hi)); the three products hi.hi + hi.lo + lo.hi
// accumulate in FP32 in tensor memory, which keeps about 16 significant bits
// of every product.  One persistent CTA of six warps per SM computes 128 x 256
// tiles with a warp-specialised four-stage pipeline: one thread of warp 0 issues
// TMA loads of 32-wide K slices (64-byte swizzled shared memory, completion counted in
// bytes on a per-stage mbarrier), one thread of warp 1 issues tcgen05.mma into one
// of two 256-column tensor-memory accumulators and commits each stage back to the
// producer, and the four epilogue warps read the other accumulator's 32 lanes each
// back with tcgen05.ld, so a tile's epilogue overlaps the next tile's products.
// Every mbarrier wait is bounded; a wait that gives up sets an error word that
// the host reads.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/hobc_tc.h"
#include "hobc_internal.h"
#include "hobc_kernels.cuh"

namespace hobc {
namespace tc {

constexpr int BM = 128;          // tile rows (accumulator lanes)
constexpr int BN = 256;          // tile columns (accumulator columns)
constexpr int BK = 32;           // K per stage: one 64-byte swizzled row per operand row
constexpr int STAGES = 4;
constexpr int THREADS = 192;     // warp 0: TMA producer, warp 1: MMA issuer, warps 2-5: epilogue
constexpr int ACC = 2;           // accumulators in tensor memory (epilogue of one tile overlaps the next)
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;     // A hi, A lo, B hi, B lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 1024;   // + alignment slack, barriers, TMEM slot
constexpr unsigned WAIT_LIMIT = 1u << 22;                  // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of a K-major tile in the 64-byte swizzled
// layout TMA writes: rows of 64 bytes, 8-row groups 512 bytes apart (the
// stride field); the leading field is not used by this layout.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;                     // leading byte offset (unused): 16 bytes
    d |= (uint64_t)(512u >> 4) << 32;            // stride byte offset: 512
    d |= (uint64_t)1u << 46;                     // descriptor version of this architecture family
    d |= (uint64_t)4u << 61;                     // layout: 64-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M in units of 8 and 16.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for phase `parity` of an mbarrier; false if it gave up.
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity) {
    for (unsigned it = 0; it < WAIT_LIMIT; ++it)
        if (try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 2D TMA load of box (x = K offset, y = row) into shared memory, completing on bar.
__device__ __forceinline__ void tma_load(uint32_t sdst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(sdst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

struct Maps {                    // tensor maps of the four operand arrays
    CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

struct Output {
    int mode;                    // HOBC_TC_OUT_*
    float* f32;                  // FP32 output
    __nv_bfloat16* hi;           // split output
    __nv_bfloat16* lo;
    long long ld;                // elements between output rows
    long long batch_stride;
    int rows, cols;              // valid extent (M, N) of C
};

__device__ __forceinline__ void split_store(__nv_bfloat16* hi, __nv_bfloat16* lo, long long idx, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[idx] = h;
    lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Persistent: CTA c takes tiles c, c + gridDim.x, ... of the ntn x ntm x batch
// tiles (N tile fastest).  Rows of problem z start at z * a_rpp (A) and
// z * b_rpp (B) in the maps' row space.  Stage barriers full/empty pace the
// producer and the MMA thread; accumulator barriers tfull/tempty pace the
// MMA thread and the four epilogue warps.
__global__ void __launch_bounds__(THREADS, 1)
k_gemm_split(const __grid_constant__ Maps maps, int a_rpp, int b_rpp, int KT, int ntn, int ntm, int ntiles,
             Output out, int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    // swizzled tiles want 1024-byte alignment
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + ACC;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + ACC);
    int* progress = reinterpret_cast<int*>(tmem_slot + 1);         // [0] stages loaded, [1] stages consumed
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ACC * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(1));
        }
        for (int a = 0; a < ACC; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tfull[a])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tempty[a])), "r"(4));
        }
        progress[0] = 0;
        progress[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("fence.proxy.async.shared::cta;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (threadIdx.x == 0) {                      // producer: TMA loads of every K slice of every tile
        int it = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int nt = t % ntn, rest = t / ntn, mt = rest % ntm, z = rest / ntm;
            const int ya = z * a_rpp + mt * BM, yb = z * b_rpp + nt * BN;
            for (int kt = 0; kt < KT; ++kt, ++it) {
                const int s = it % STAGES;
                if (it >= STAGES && !wait_bounded(&empty[s], (uint32_t)((it / STAGES - 1) & 1))) { ok = false; break; }
                const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                expect_tx(&full[s], STAGE_BYTES);
                tma_load(sa, &maps.a_hi, kt * BK, ya, &full[s]);
                tma_load(sa + A_BYTES, &maps.a_lo, kt * BK, ya, &full[s]);
                tma_load(sa + 2 * A_BYTES, &maps.b_hi, kt * BK, yb, &full[s]);
                tma_load(sa + 2 * A_BYTES + B_BYTES, &maps.b_lo, kt * BK, yb, &full[s]);
            }
        }
        progress[0] = it;
    } else if (threadIdx.x == 32) {              // MMA issuer
        const uint32_t idesc = instr_desc(BM, BN);
        int it = 0, tc_ = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tc_) {
            const int a = tc_ % ACC;
            if (tc_ >= ACC && !wait_bounded(&tempty[a], (uint32_t)((tc_ / ACC - 1) & 1))) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t acc = tmem + (uint32_t)(a * BN);
            for (int kt = 0; kt < KT; ++kt, ++it) {
                const int s = it % STAGES;
                if (!wait_bounded(&full[s], (uint32_t)((it / STAGES) & 1))) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                const uint32_t a_hi = sa, a_lo = sa + A_BYTES, b_hi = sa + 2 * A_BYTES, b_lo = b_hi + B_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint32_t ko = kk * 32;         // 16 bf16 of K inside the 64-byte row
                    const uint64_t dah = smem_desc_sw64(a_hi + ko), dal = smem_desc_sw64(a_lo + ko);
                    const uint64_t dbh = smem_desc_sw64(b_hi + ko), dbl = smem_desc_sw64(b_lo + ko);
                    mma(acc, dah, dbh, idesc, (kt | kk) ? 1u : 0u);
                    mma(acc, dah, dbl, idesc, 1u);
                    mma(acc, dal, dbh, idesc, 1u);
                }
                commit(&empty[s]);
            }
            if (!ok) break;
            commit(&tfull[a]);
        }
        progress[1] = it;
    } else if (warp >= 2) {                      // epilogue: accumulator lanes of quarter warp % 4
        const int q = warp % 4;
        int tc_ = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc_) {
            const int a = tc_ % ACC;
            if (!wait_bounded(&tfull[a], (uint32_t)((tc_ / ACC) & 1))) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int nt = t % ntn, rest = t / ntn, mt = rest % ntm, z = rest / ntm;
            const int row = mt * BM + q * 32 + lane, n0 = nt * BN;
            const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN);
            const long long zb = (long long)z * out.batch_stride;
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(base + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < out.rows) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = n0 + c0 + j;
                        if (col >= out.cols) break;
                        const float v = __uint_as_float(r[j]);
                        if (out.mode == HOBC_TC_OUT_F32) {
                            out.f32[zb + (long long)row * out.ld + col] = v;
                        } else if (out.mode == HOBC_TC_OUT_F32_T) {
                            out.f32[zb + (long long)col * out.ld + row] = v;
                        } else if (out.mode == HOBC_TC_OUT_SPLIT) {
                            split_store(out.hi, out.lo, zb + (long long)row * out.ld + col, v);
                        } else {
                            split_store(out.hi, out.lo, zb + (long long)col * out.ld + row, v);
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[a])) : "memory");
        }
    }
    if (!ok && lane == 0) atomicOr(err, 1);
    __syncthreads();
    if (threadIdx.x == 0) {                      // let loads still in flight land before the CTA exits
        for (int it = progress[1]; it < progress[0]; ++it)
            wait_bounded(&full[it % STAGES], (uint32_t)((it / STAGES) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ACC * BN));
}

// x -> (bf16(x), bf16(x - bf16(x))) into a zero-padded K-major layout: source
// [batch][rows][cols] (row stride src_ld) to [batch][rows_p][ld] (cols_p = ld).
__global__ void k_split(const float* __restrict__ src, long long src_ld, long long src_bs, int rows, int cols,
                        __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long long ld,
                        long long bs, int rows_p, int batch) {
    const long long per = (long long)rows_p * ld;
    const long long total = per * batch;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / per, rem = i - b * per;
        const int r = (int)(rem / ld), c = (int)(rem - (long long)r * ld);
        const float v = (r < rows && c < cols) ? src[b * src_bs + (long long)r * src_ld + c] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[b * bs + (long long)r * ld + c] = h;
        lo[b * bs + (long long)r * ld + c] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// src holds a matrix transposed (FP64, src[c][r] at c * src_ld + r); write
// rows r < rows, columns c < cols of its transpose as a split operand.
__global__ void k_split_f64_t(const double* __restrict__ src, long long src_ld, int rows, int cols,
                              __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long long ld) {
    const long long total = (long long)rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i - (long long)r * cols);
        const double v = src[(long long)c * src_ld + r];
        const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
        hi[(long long)r * ld + c] = h;
        lo[(long long)r * ld + c] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
    }
}

// Row-major FP64 matrix (src[r][c] at r * src_ld + c) -> split operand rows r < rows,
// columns c < cols.
__global__ void k_split_f64(const double* __restrict__ src, long long src_ld, int rows, int cols,
                            __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long long ld) {
    const long long total = (long long)rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i - (long long)r * cols);
        const double v = src[(long long)r * src_ld + c];
        const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
        hi[(long long)r * ld + c] = h;
        lo[(long long)r * ld + c] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
    }
}

// Filter (Eq. (eq:freg)) of the spectrum and split into the A operand of the
// first synthesis pass.  2D: spectrum [item][t1][t0] -> rows t1, columns t0;
// 1D: [item][t] -> row item, column t.  fd.D null: no filter (plain synthesis).
__global__ void k_filter_split(const float* __restrict__ spec, long long S, int nrows, int ncols, int ndim,
                               Axis<float> ax0, FilterDesc fd, int items, __nv_bfloat16* __restrict__ hi,
                               __nv_bfloat16* __restrict__ lo, long long ld, long long bs) {
    const long long per = (long long)nrows * ncols;
    const long long total = per * items;
    const float* D = static_cast<const float*>(fd.D);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long item = i / per, e = i - item * per;
        const int r = (int)(e / ncols), c = (int)(e - (long long)r * ncols);
        float v = spec[item * S + e];
        if (D) {
            const int problem = (int)item;
            const float d = D[(fd.psf_per ? item : 0) * fd.d_psf_stride + e];
            const float s2 = smoothing2<float>(fd, ndim == 2 ? 2 : 1, ax0, ndim == 2 ? r : problem, c);
            v = apply_filter(v, d, s2, (float)mu_of(fd, problem));
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const long long o = ndim == 2 ? item * bs + (long long)r * ld + c : (item) * ld + c;
        hi[o] = h;
        lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// Fourier family: filter (Eq. (eq:freg), complex) of the half spectrum and
// split, re and im interleaved along K.  2D: spectrum [item][c][t0] -> rows c,
// columns 2 t0 + part; 1D: [item][c] -> row item, columns 2 c + part.
// fd.D null: no filter (plain synthesis).
__global__ void k_filter_split_cplx(const float2* __restrict__ spec, long long S, int nrows, int ncols, int ndim,
                                    Axis<float> ax0, FilterDesc fd, int items, __nv_bfloat16* __restrict__ hi,
                                    __nv_bfloat16* __restrict__ lo, long long ld, long long bs) {
    const long long per = (long long)nrows * ncols;
    const long long total = per * items;
    const float2* D = static_cast<const float2*>(fd.D);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long item = i / per, e = i - item * per;
        const int r = (int)(e / ncols), c = (int)(e - (long long)r * ncols);
        float2 v = spec[item * S + e];
        if (D) {
            const int problem = (int)item;
            const float2 d = D[(fd.psf_per ? item : 0) * fd.d_psf_stride + e];
            const float s2 = smoothing2<float>(fd, ndim == 2 ? 2 : 1, ax0, ndim == 2 ? r : problem, c);
            v = apply_filter(v, d, s2, (float)mu_of(fd, problem));
        }
        const long long o = ndim == 2 ? item * bs + (long long)r * ld + 2 * c : item * ld + 2 * c;
        const __nv_bfloat16 hx = __float2bfloat16_rn(v.x), hy = __float2bfloat16_rn(v.y);
        hi[o] = hx;
        lo[o] = __float2bfloat16_rn(v.x - __bfloat162float(hx));
        hi[o + 1] = hy;
        lo[o + 1] = __float2bfloat16_rn(v.y - __bfloat162float(hy));
    }
}

// ------------------------------------------------------------ tensor maps

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiled g_encode = nullptr;

hobc_status encode_maps() {
    if (g_encode) return HOBC_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        set_last_error_text("hobc_tc_gemm: cuTensorMapEncodeTiled is not available");
        return HOBC_ERR_CUDA;
    }
    g_encode = reinterpret_cast<EncodeTiled>(fn);
    return HOBC_OK;
}

// Rows x K bf16 array (row stride ld elements) read in boxes of BK x box_rows,
// 64-byte swizzled; reads outside the array return zeros.
hobc_status make_map(CUtensorMap* map, const void* base, long long k, long long ld, long long rows, int box_rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char msg[96];
        snprintf(msg, sizeof(msg), "hobc_tc_gemm: cuTensorMapEncodeTiled failed (%d)", (int)r);
        set_last_error_text(msg);
        return HOBC_ERR_ARG;
    }
    return HOBC_OK;
}

}  // namespace tc
}  // namespace hobc

using namespace hobc;

// ===================================================== dense plan (HOBC_SPLIT_BF16)

struct hobc_dense_s {
    int nax;
    int n[2];
    long long kp[2];                       // padded K per axis
    // split matrices: 2D 0 = T1^{-1} (B), 1 = T0^{-1} (A), 2 = T0 (B), 3 = T1 (A);
    //                 1D 0 = T^{-1} (B), 2 = T (B)
    __nv_bfloat16* m_hi[4];
    __nv_bfloat16* m_lo[4];
    long long m_ld[4];
    // operand workspace: 0 = g (A), 1 = row-pass output (B), 2 = filtered spectrum (A), 3 = column-synthesis output (B)
    __nv_bfloat16* w_hi[4];
    __nv_bfloat16* w_lo[4];
    long long w_ld[4], w_bs[4];
    int* err;
    // Fourier family: stored columns of the last axis and the padded K of its
    // (c, part) pairs (kw per part), and the padded K of axis 0's (t0, part) pairs
    int fourier, W;
    long long kw, k2;
};

namespace {

long long pad_to(long long x, long long t) { return (x + t - 1) / t * t; }

hobc_status gemm(hobc_plan_s* p, const __nv_bfloat16* ah, const __nv_bfloat16* al, long long ald, long long abs_,
                 const __nv_bfloat16* bh, const __nv_bfloat16* bl, long long bld, long long bbs, int m, int n, long long k,
                 int batch, int mode, float* f32, __nv_bfloat16* oh, __nv_bfloat16* ol, long long old_, long long obs) {
    hobc_tc_operand A{ah, al, ald, abs_};
    hobc_tc_operand B{bh, bl, bld, bbs};
    hobc_tc_output O{mode, f32, oh, ol, old_, obs, m, n};
    hobc_status s = hobc_tc_gemm(&A, &B, m, n, (int)k, batch, &O, p->dense->err, p->stream);
    if (s == HOBC_OK) ++p->launches;
    return s;
}

Axis<float> axis0(const hobc_plan_s* p) {
    Axis<float> a;
    memset(&a, 0, sizeof(a));
    a.fam = p->ax[0].fam; a.n = p->ax[0].n; a.N = p->ax[0].N; a.W = p->ax[0].W;
    return a;
}

FilterDesc filter_desc(const hobc_plan_s* p, const void* D, const int* mu_idx, const double* mu_val) {
    FilterDesc f;
    memset(&f, 0, sizeof(f));
    f.D = D;
    f.d_psf_stride = (long long)p->spec_elems;
    f.psf_per = p->desc.psf_per_item;
    f.mu_idx = mu_idx;
    f.mu = p->mu;
    f.K = p->K;
    f.lap = p->desc.L == HOBC_L_LAPLACIAN;
    const AxisHost& o = p->ax[p->nax - 1];
    f.o_fam = o.fam; f.o_n = o.n; f.o_N = o.N; f.o_W = o.W;
    f.mu_val = mu_val;
    return f;
}

hobc_status check(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error(what, e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

// Synthesis from the split operand already in workspace 2 (rows of the filtered spectrum).
hobc_status dense_synthesis_from_x(hobc_plan_s* p, float* y) {
    hobc_dense_s* d = p->dense;
    const int B = p->desc.batch;
    const size_t z0 = p->item0;
    if (d->nax == 1) {
        const int n = d->n[0];
        return gemm(p, d->w_hi[2] + z0 * d->w_ld[2], d->w_lo[2] + z0 * d->w_ld[2], d->w_ld[2], 0, d->m_hi[2],
                    d->m_lo[2], d->m_ld[2], 0, B, n, d->kp[0], 1, HOBC_TC_OUT_F32, y, nullptr, nullptr, n, 0);
    }
    const int n0 = d->n[0], n1 = d->n[1];
    // columns: Y[t1][r] = sum_t0 X[t1][t0] T0[r][t0], stored transposed (rows r)
    hobc_status s = gemm(p, d->w_hi[2] + z0 * d->w_bs[2], d->w_lo[2] + z0 * d->w_bs[2], d->w_ld[2], d->w_bs[2],
                         d->m_hi[2], d->m_lo[2], d->m_ld[2], 0, n1, n0, d->kp[0], B, HOBC_TC_OUT_SPLIT_T, nullptr,
                         d->w_hi[3] + z0 * d->w_bs[3], d->w_lo[3] + z0 * d->w_bs[3], d->w_ld[3], d->w_bs[3]);
    if (s != HOBC_OK) return s;
    // rows: f[r][j] = sum_t1 T1[j][t1] Y[t1][r], computed as C[j][r] and stored transposed
    return gemm(p, d->m_hi[3], d->m_lo[3], d->m_ld[3], 0, d->w_hi[3] + z0 * d->w_bs[3], d->w_lo[3] + z0 * d->w_bs[3],
                d->w_ld[3], d->w_bs[3], n1, n0, d->kp[1], B, HOBC_TC_OUT_F32_T, y, nullptr, nullptr, n1,
                (long long)n0 * n1);
}

}  // namespace

namespace hobc {

// Responses of the FP64 path of a 1D Fourier axis of n samples to unit inputs:
// A[j][c] (complex, W per j) = analysis of the real unit e_j, i.e. T^{-1}[t(c)][j];
// Y[u][i] (n per u) = synthesis of the half spectrum with a real (u = 2c) or
// imaginary (u = 2c + 1) unit at stored entry c.
static hobc_status fourier_unit_responses(int n, cudaStream_t st, std::vector<double>& A, std::vector<double>& Y) {
    const int N = n - 2, W = N / 2 + 3;
    const int items = std::max(n, 2 * W);
    hobc_plan_desc q;
    memset(&q, 0, sizeof(q));
    q.ndim = 1; q.n[0] = n; q.psf[0] = 1; q.family = HOBC_FAMILY_FOURIER; q.bc_degree = 2;
    q.L = HOBC_L_IDENTITY; q.prec = HOBC_FP64; q.n_mu = 1; q.batch = items; q.psf_per_item = 0;
    const double one = 1.0;
    hobc_plan* ip = nullptr;
    hobc_status s = hobc_plan_create(&q, &one, st, &ip);
    if (s != HOBC_OK) return s;
    std::vector<double> in_real((size_t)items * n, 0.0), in_spec((size_t)items * 2 * W, 0.0);
    for (int j = 0; j < n; ++j) in_real[(size_t)j * n + j] = 1.0;
    for (int u = 0; u < 2 * W; ++u) in_spec[(size_t)u * 2 * W + u] = 1.0;     // item u: unit at (c, part) = u
    double *dr = nullptr, *ds = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc((void**)&dr, in_real.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ds, in_spec.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&dout, (size_t)items * std::max(n, 2 * W) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(dr, in_real.data(), in_real.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ds, in_spec.data(), in_spec.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) s = hobc_analysis(ip, dr, dout);
    if (e == cudaSuccess && s == HOBC_OK) e = cudaStreamSynchronize(st);
    A.assign((size_t)n * 2 * W, 0.0);
    if (e == cudaSuccess && s == HOBC_OK) e = cudaMemcpy(A.data(), dout, A.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && s == HOBC_OK) s = hobc_synthesis(ip, ds, dout);
    if (e == cudaSuccess && s == HOBC_OK) e = cudaStreamSynchronize(st);
    Y.assign((size_t)2 * W * n, 0.0);
    if (e == cudaSuccess && s == HOBC_OK) e = cudaMemcpy(Y.data(), dout, Y.size() * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(dr);
    cudaFree(ds);
    cudaFree(dout);
    hobc_plan_destroy(ip);
    if (s != HOBC_OK) return s;
    if (e != cudaSuccess) { set_last_error("hobc_plan_create (dense Fourier matrices)", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

// Dense split-BF16 mode of the Fourier family (real arithmetic on the tensor
// cores).  Each complex product is a real GEMM on (re, im) pairs:
//   2D analysis   rows: C[r][2c+p]  = g[r][:] . M1a[2c+p][:],   M1a = (Re, Im) of T1^{-1} on the stored half;
//                 stored transposed, so row c of the result holds (Re | Im) of column c over r;
//                 columns: ghat[c][2t0+p] = [Re | Im](c) . M0a[2t0+p][:], M0a the real form of T0^{-1};
//   2D synthesis  columns: Y[2r+p][c] = M0s[2r+p][:] . X[c][:] (X interleaved (t0, part)), M0s the real
//                 form of T0; rows 2r, 2r+1 of Y read as one row of (Re | Im) over c;
//                 rows: f[r][j] = M1s[j][:] . Y(r), M1s[j][(p, c)] the FP64 synthesis of a unit at (c, p);
//   1D            the last-axis products alone, with K interleaved (c, part).
// The matrices are the FP64 path's own responses to unit inputs (fourier_unit_responses).
static hobc_status dense_prepare_fourier(hobc_plan_s* p) {
    hobc_dense_s* d = p->dense;
    d->fourier = 1;
    const int B = p->desc.batch;
    const int nl = d->n[p->nax - 1];
    const int W = p->ax[p->nax - 1].W;
    d->W = W;
    cudaError_t e = cudaSuccess;
    auto alloc2 = [&](__nv_bfloat16** hi, __nv_bfloat16** lo, size_t elems) {
        if (e == cudaSuccess) e = cudaMalloc((void**)hi, elems * 2);
        if (e == cudaSuccess) e = cudaMalloc((void**)lo, elems * 2);
        if (e == cudaSuccess) e = cudaMemset(*hi, 0, elems * 2);
        if (e == cudaSuccess) e = cudaMemset(*lo, 0, elems * 2);
    };
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d->err, 0, sizeof(int));
    const long long kl = d->kp[p->nax - 1];                  // K of the last axis (samples j)
    d->kw = pad_to(W, tc::BK);
    std::vector<std::vector<double>> host(4);
    std::vector<int> mrows(4, 0), mcols(4, 0);
    // last axis: analysis rows (2c + p) over j; synthesis columns over (c, p)
    std::vector<double> A1, Y1;
    hobc_status s = fourier_unit_responses(nl, p->stream, A1, Y1);
    if (s != HOBC_OK) return s;
    {
        const long long rows = pad_to(2 * W, tc::BN);
        d->m_ld[0] = kl;
        alloc2(&d->m_hi[0], &d->m_lo[0], (size_t)rows * kl);
        host[0].assign((size_t)2 * W * nl, 0.0);
        for (int c = 0; c < W; ++c)
            for (int j = 0; j < nl; ++j) {
                host[0][(size_t)(2 * c) * nl + j] = A1[((size_t)j * W + c) * 2];
                host[0][(size_t)(2 * c + 1) * nl + j] = A1[((size_t)j * W + c) * 2 + 1];
            }
        mrows[0] = 2 * W; mcols[0] = nl;
    }
    if (p->nax == 1) {
        // synthesis: f[item][j] = X[item][2c + p] . M[j][2c + p]
        d->k2 = pad_to(2 * W, tc::BK);
        const long long rows = pad_to(nl, tc::BN);
        d->m_ld[2] = d->k2;
        alloc2(&d->m_hi[2], &d->m_lo[2], (size_t)rows * d->k2);
        host[2].assign((size_t)nl * 2 * W, 0.0);
        for (int j = 0; j < nl; ++j)
            for (int u = 0; u < 2 * W; ++u) host[2][(size_t)j * 2 * W + u] = Y1[(size_t)u * nl + j];
        mrows[2] = nl; mcols[2] = 2 * W;
        const long long wrows = pad_to(B, tc::BM) + tc::BM;   // a chunk's last tile may run past the batch
        d->w_ld[0] = kl; d->w_bs[0] = 0;
        alloc2(&d->w_hi[0], &d->w_lo[0], (size_t)wrows * kl);
        d->w_ld[2] = d->k2; d->w_bs[2] = 0;
        alloc2(&d->w_hi[2], &d->w_lo[2], (size_t)wrows * d->k2);
    } else {
        const int n0 = d->n[0], n1 = d->n[1];
        const long long k0 = d->kp[0];
        d->k2 = pad_to(2 * n0, tc::BK);
        // synthesis rows: M1s[j][p * kw + c] = Y1[2c + p][j]
        {
            const long long rows = pad_to(n1, tc::BM);
            d->m_ld[3] = 2 * d->kw;
            alloc2(&d->m_hi[3], &d->m_lo[3], (size_t)rows * 2 * d->kw);
            host[3].assign((size_t)n1 * 2 * d->kw, 0.0);
            for (int j = 0; j < n1; ++j)
                for (int c = 0; c < W; ++c)
                    for (int pp = 0; pp < 2; ++pp)
                        host[3][(size_t)j * 2 * d->kw + pp * d->kw + c] = Y1[(size_t)(2 * c + pp) * n1 + j];
            mrows[3] = n1; mcols[3] = (int)(2 * d->kw);
        }
        // axis 0: the full complex T0^{-1} and T0 from the unit responses of a 1D axis of n0
        std::vector<double> A0, Y0;
        s = fourier_unit_responses(n0, p->stream, A0, Y0);
        if (s != HOBC_OK) return s;
        const int N0 = n0 - 2, W0 = N0 / 2 + 3;
        auto t_of = [&](int c) { return c == W0 - 1 ? n0 - 1 : c; };
        auto self_of = [&](int c) { return c == 0 || c == W0 - 1 || c == 1 || 2 * (c - 1) == N0; };
        auto neg = [&](int t) { return (t == 0 || t == n0 - 1) ? t : 1 + (N0 - (t - 1)) % N0; };
        std::vector<double> Tir((size_t)n0 * n0), Tii((size_t)n0 * n0), Tr((size_t)n0 * n0), Ti((size_t)n0 * n0);
        for (int c = 0; c < W0; ++c) {
            const int t = t_of(c), tn = neg(t);
            for (int r = 0; r < n0; ++r) {
                const double re = A0[((size_t)r * W0 + c) * 2], im = A0[((size_t)r * W0 + c) * 2 + 1];
                Tir[(size_t)t * n0 + r] = re; Tii[(size_t)t * n0 + r] = im;           // T0^{-1}[t][r]
                if (!self_of(c)) { Tir[(size_t)tn * n0 + r] = re; Tii[(size_t)tn * n0 + r] = -im; }
                const double yr = Y0[(size_t)(2 * c) * n0 + r], yi = Y0[(size_t)(2 * c + 1) * n0 + r];
                if (self_of(c)) {
                    Tr[(size_t)r * n0 + t] = yr; Ti[(size_t)r * n0 + t] = 0.0;         // T0[r][t]
                } else {
                    Tr[(size_t)r * n0 + t] = 0.5 * yr; Ti[(size_t)r * n0 + t] = -0.5 * yi;
                    Tr[(size_t)r * n0 + tn] = 0.5 * yr; Ti[(size_t)r * n0 + tn] = 0.5 * yi;
                }
            }
        }
        // analysis columns: M0a[2t0 + po][pi * k0 + r]
        {
            const long long rows = pad_to(2 * n0, tc::BN);
            d->m_ld[1] = 2 * k0;
            alloc2(&d->m_hi[1], &d->m_lo[1], (size_t)rows * 2 * k0);
            host[1].assign((size_t)2 * n0 * 2 * k0, 0.0);
            for (int t = 0; t < n0; ++t)
                for (int r = 0; r < n0; ++r) {
                    const double re = Tir[(size_t)t * n0 + r], im = Tii[(size_t)t * n0 + r];
                    double* row0 = &host[1][(size_t)(2 * t) * 2 * k0];
                    double* row1 = &host[1][(size_t)(2 * t + 1) * 2 * k0];
                    row0[r] = re; row0[k0 + r] = -im;
                    row1[r] = im; row1[k0 + r] = re;
                }
            mrows[1] = 2 * n0; mcols[1] = (int)(2 * k0);
        }
        // synthesis columns: M0s[2r + po][2t0 + pi]
        {
            const long long rows = pad_to(2 * n0, tc::BM);
            d->m_ld[2] = d->k2;
            alloc2(&d->m_hi[2], &d->m_lo[2], (size_t)rows * d->k2);
            host[2].assign((size_t)2 * n0 * d->k2, 0.0);
            for (int r = 0; r < n0; ++r)
                for (int t = 0; t < n0; ++t) {
                    const double re = Tr[(size_t)r * n0 + t], im = Ti[(size_t)r * n0 + t];
                    double* row0 = &host[2][(size_t)(2 * r) * d->k2];
                    double* row1 = &host[2][(size_t)(2 * r + 1) * d->k2];
                    row0[2 * t] = re; row0[2 * t + 1] = -im;
                    row1[2 * t] = im; row1[2 * t + 1] = re;
                }
            mrows[2] = 2 * n0; mcols[2] = (int)d->k2;
        }
        // operand workspace (per problem)
        const long long r0 = pad_to(n0, tc::BM), rw = pad_to(W, tc::BM), rwb = pad_to(W, tc::BN), r0b = pad_to(n0, tc::BN);
        d->w_ld[0] = kl;          d->w_bs[0] = r0 * kl;              // g split (A)
        d->w_ld[1] = 2 * k0;      d->w_bs[1] = rw * 2 * k0;          // row-pass output, read as [c][(p, r)] (A)
        d->w_ld[2] = d->k2;       d->w_bs[2] = rwb * d->k2;          // filtered spectrum [c][(t0, p)] (B)
        d->w_ld[3] = 2 * d->kw;   d->w_bs[3] = r0b * 2 * d->kw;      // column-synthesis output, read as [r][(p, c)] (B)
        for (int w = 0; w < 4; ++w) alloc2(&d->w_hi[w], &d->w_lo[w], (size_t)B * d->w_bs[w]);
    }
    if (e != cudaSuccess) { set_last_error("hobc_plan_create (dense)", e); return HOBC_ERR_CUDA; }
    for (int m = 0; m < 4 && e == cudaSuccess; ++m) {
        if (host[m].empty()) continue;
        double* dev = nullptr;
        e = cudaMalloc((void**)&dev, host[m].size() * sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(dev, host[m].data(), host[m].size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            tc::k_split_f64<<<1024, 256, 0, p->stream>>>(dev, mcols[m], mrows[m], mcols[m], d->m_hi[m], d->m_lo[m],
                                                         d->m_ld[m]);
            e = cudaStreamSynchronize(p->stream);
        }
        cudaFree(dev);
    }
    if (e != cudaSuccess) { set_last_error("hobc_plan_create (dense)", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

void dense_free(hobc_plan_s* p) {
    hobc_dense_s* d = p->dense;
    if (!d) return;
    for (int i = 0; i < 4; ++i) {
        cudaFree(d->m_hi[i]); cudaFree(d->m_lo[i]); cudaFree(d->w_hi[i]); cudaFree(d->w_lo[i]);
    }
    cudaFree(d->err);
    delete d;
    p->dense = nullptr;
}

hobc_status dense_prepare(hobc_plan_s* p) {
    hobc_dense_s* d = new hobc_dense_s();
    p->dense = d;
    d->nax = p->nax;
    const int B = p->desc.batch;
    for (int a = 0; a < p->nax; ++a) {
        d->n[a] = p->ax[a].n;
        d->kp[a] = pad_to(d->n[a], tc::BK);
    }
    if (p->fam == HOBC_FAMILY_FOURIER) return dense_prepare_fourier(p);
    cudaError_t e = cudaSuccess;
    auto alloc2 = [&](__nv_bfloat16** hi, __nv_bfloat16** lo, size_t elems) {
        if (e == cudaSuccess) e = cudaMalloc((void**)hi, elems * 2);
        if (e == cudaSuccess) e = cudaMalloc((void**)lo, elems * 2);
        if (e == cudaSuccess) e = cudaMemset(*hi, 0, elems * 2);
        if (e == cudaSuccess) e = cudaMemset(*lo, 0, elems * 2);
    };
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d->err, 0, sizeof(int));
    // the matrices: T_X and T_X^{-1} of each axis from the FP64 path applied to identities
    int mi[2][2];                      // matrix slot of (axis, inverse?)
    if (p->nax == 2) { mi[1][1] = 0; mi[0][1] = 1; mi[0][0] = 2; mi[1][0] = 3; }
    else { mi[0][1] = 0; mi[0][0] = 2; }
    for (int a = 0; a < p->nax && e == cudaSuccess; ++a) {
        const int n = d->n[a];
        const long long kp = d->kp[a];
        for (int inv = 0; inv < 2 && e == cudaSuccess; ++inv) {
            const int slot = mi[a][inv];
            const bool as_a = p->nax == 2 && (slot == 1 || slot == 3);
            const long long rows = pad_to(n, as_a ? tc::BM : tc::BN);
            d->m_ld[slot] = kp;
            alloc2(&d->m_hi[slot], &d->m_lo[slot], (size_t)rows * kp);
        }
    }
    // operand workspace
    if (p->nax == 2) {
        const long long n0 = d->n[0], n1 = d->n[1];
        const long long rows[4] = {pad_to(n0, tc::BM), pad_to(n1, tc::BN), pad_to(n1, tc::BM), pad_to(n0, tc::BN)};
        const long long lds[4] = {d->kp[1], d->kp[0], d->kp[0], d->kp[1]};
        for (int w = 0; w < 4; ++w) {
            d->w_ld[w] = lds[w];
            d->w_bs[w] = rows[w] * lds[w];
            alloc2(&d->w_hi[w], &d->w_lo[w], (size_t)B * rows[w] * lds[w]);
        }
    } else {
        const long long rows = pad_to(B, tc::BM) + tc::BM;   // a chunk's last tile may run past the batch
        for (int w : {0, 2}) {
            d->w_ld[w] = d->kp[0];
            d->w_bs[w] = 0;
            alloc2(&d->w_hi[w], &d->w_lo[w], (size_t)rows * d->kp[0]);
        }
    }
    if (e != cudaSuccess) { set_last_error("hobc_plan_create (dense)", e); return HOBC_ERR_CUDA; }
    // build T and T^{-1}
    if (p->fam == HOBC_FAMILY_REFLECTIVE || p->fam == HOBC_FAMILY_PERIODIC) {
        // the classical conditions: orthonormal C (T^{-1} = C, T = C^T) or the
        // symmetric Hartley matrix (T = T^{-1} = H), written straight from their definitions
        for (int a = 0; a < p->nax; ++a) {
            const int n = d->n[a];
            std::vector<double> X((size_t)n * n);          // X[k][j]
            for (int k = 0; k < n; ++k)
                for (int j = 0; j < n; ++j) {
                    if (p->fam == HOBC_FAMILY_REFLECTIVE) {
                        const double sc = std::sqrt((k == 0 ? 1.0 : 2.0) / n);
                        X[(size_t)k * n + j] = sc * std::cos(M_PI * k * (2.0 * j + 1.0) / (2.0 * n));
                    } else {
                        const long long r = (long long)k * j % n;
                        const double ang = 2.0 * M_PI * (double)r / n;
                        X[(size_t)k * n + j] = (std::cos(ang) + std::sin(ang)) / std::sqrt((double)n);
                    }
                }
            double* dev = nullptr;
            e = cudaMalloc((void**)&dev, X.size() * sizeof(double));
            for (int inv = 1; inv >= 0 && e == cudaSuccess; --inv) {
                // k_split_f64_t writes the transpose of what it reads: feed it the
                // transpose of the wanted matrix (T^{-1} = X, T = X^T)
                std::vector<double> src((size_t)n * n);
                for (int r = 0; r < n; ++r)
                    for (int c = 0; c < n; ++c)
                        src[(size_t)c * n + r] = inv ? X[(size_t)r * n + c] : X[(size_t)c * n + r];
                e = cudaMemcpy(dev, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice);
                if (e != cudaSuccess) break;
                const int slot = mi[a][inv];
                tc::k_split_f64_t<<<256, 256, 0, p->stream>>>(dev, n, n, n, d->m_hi[slot], d->m_lo[slot],
                                                               d->m_ld[slot]);
                e = cudaStreamSynchronize(p->stream);
            }
            cudaFree(dev);
            if (e != cudaSuccess) { set_last_error("hobc_plan_create (dense)", e); return HOBC_ERR_CUDA; }
        }
        return HOBC_OK;
    }
    for (int a = 0; a < p->nax; ++a) {
        const int n = d->n[a];
        hobc_plan_desc q;
        memset(&q, 0, sizeof(q));
        q.ndim = 1; q.n[0] = n; q.psf[0] = 1; q.family = (hobc_family)p->fam; q.psf_symmetric = 1;
        q.bc_degree = p->fam == HOBC_FAMILY_SINE ? 1 : (p->fam == HOBC_FAMILY_COSINE ? 2 : 3);
        q.L = HOBC_L_IDENTITY; q.prec = HOBC_FP64; q.n_mu = 1; q.batch = n; q.psf_per_item = 0;
        const double one = 1.0;
        hobc_plan* ip = nullptr;
        hobc_status s = hobc_plan_create(&q, &one, p->stream, &ip);
        if (s != HOBC_OK) return s;
        double *I = nullptr, *out = nullptr;
        e = cudaMalloc((void**)&I, (size_t)n * n * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void**)&out, (size_t)n * n * sizeof(double));
        if (e == cudaSuccess) {
            std::vector<double> eye((size_t)n * n, 0.0);
            for (int i = 0; i < n; ++i) eye[(size_t)i * n + i] = 1.0;
            e = cudaMemcpy(I, eye.data(), eye.size() * sizeof(double), cudaMemcpyHostToDevice);
        }
        for (int inv = 1; inv >= 0 && e == cudaSuccess && s == HOBC_OK; --inv) {
            // analysis of e_j gives row j = column j of T^{-1}; synthesis of e_t gives column t of T
            s = inv ? hobc_analysis(ip, I, out) : hobc_synthesis(ip, I, out);
            if (s != HOBC_OK) break;
            const int slot = mi[a][inv];
            tc::k_split_f64_t<<<256, 256, 0, p->stream>>>(out, n, n, n, d->m_hi[slot], d->m_lo[slot], d->m_ld[slot]);
            e = cudaStreamSynchronize(p->stream);
        }
        cudaFree(I);
        cudaFree(out);
        hobc_plan_destroy(ip);
        if (s != HOBC_OK) return s;
        if (e != cudaSuccess) { set_last_error("hobc_plan_create (dense)", e); return HOBC_ERR_CUDA; }
    }
    return HOBC_OK;
}

// Fourier family (see dense_prepare_fourier): g real -> half spectrum [c][t0] (re, im).
static hobc_status dense_analysis_fourier(hobc_plan_s* p, const float* gf, float* out) {
    hobc_dense_s* d = p->dense;
    const int B = p->desc.batch;
    const size_t z0 = p->item0;
    const int W = d->W;
    if (d->nax == 1) {
        const int n = d->n[0];
        hobc_status s = hobc_tc_split(gf, n, 0, B, n, d->w_hi[0] + z0 * d->w_ld[0], d->w_lo[0] + z0 * d->w_ld[0],
                                      d->w_ld[0], 0, B, 1, p->stream);
        if (s != HOBC_OK) return s;
        ++p->launches;
        return gemm(p, d->w_hi[0] + z0 * d->w_ld[0], d->w_lo[0] + z0 * d->w_ld[0], d->w_ld[0], 0, d->m_hi[0],
                    d->m_lo[0], d->m_ld[0], 0, B, 2 * W, d->kp[0], 1, HOBC_TC_OUT_F32, out, nullptr, nullptr, 2 * W, 0);
    }
    const int n0 = d->n[0], n1 = d->n[1];
    hobc_status s = hobc_tc_split(gf, n1, (long long)n0 * n1, n0, n1, d->w_hi[0] + z0 * d->w_bs[0],
                                  d->w_lo[0] + z0 * d->w_bs[0], d->w_ld[0], d->w_bs[0], n0, B, p->stream);
    if (s != HOBC_OK) return s;
    ++p->launches;
    // rows: C[r][2c + p] = sum_j g[r][j] M1a[2c + p][j], stored transposed: row 2c + p of length k0
    s = gemm(p, d->w_hi[0] + z0 * d->w_bs[0], d->w_lo[0] + z0 * d->w_bs[0], d->w_ld[0], d->w_bs[0], d->m_hi[0],
             d->m_lo[0], d->m_ld[0], 0, n0, 2 * W, d->kp[1], B, HOBC_TC_OUT_SPLIT_T, nullptr,
             d->w_hi[1] + z0 * d->w_bs[1], d->w_lo[1] + z0 * d->w_bs[1], d->kp[0], d->w_bs[1]);
    if (s != HOBC_OK) return s;
    // columns: ghat[c][2t0 + p] = sum_(q, r) R[c][(q, r)] M0a[2t0 + p][(q, r)]
    return gemm(p, d->w_hi[1] + z0 * d->w_bs[1], d->w_lo[1] + z0 * d->w_bs[1], d->w_ld[1], d->w_bs[1], d->m_hi[1],
                d->m_lo[1], d->m_ld[1], 0, W, 2 * n0, 2 * d->kp[0], B, HOBC_TC_OUT_F32, out, nullptr, nullptr,
                2 * n0, (long long)W * 2 * n0);
}

hobc_status dense_analysis(hobc_plan_s* p, const void* g, void* ghat) {
    hobc_dense_s* d = p->dense;
    if (d->fourier) return dense_analysis_fourier(p, static_cast<const float*>(g), static_cast<float*>(ghat));
    const int B = p->desc.batch;
    const size_t z0 = p->item0;
    const float* gf = static_cast<const float*>(g);
    float* out = static_cast<float*>(ghat);
    if (d->nax == 1) {
        const int n = d->n[0];
        hobc_status s = hobc_tc_split(gf, n, 0, B, n, d->w_hi[0] + z0 * d->w_ld[0], d->w_lo[0] + z0 * d->w_ld[0],
                                      d->w_ld[0], 0, B, 1, p->stream);
        if (s != HOBC_OK) return s;
        ++p->launches;
        return gemm(p, d->w_hi[0] + z0 * d->w_ld[0], d->w_lo[0] + z0 * d->w_ld[0], d->w_ld[0], 0, d->m_hi[0],
                    d->m_lo[0], d->m_ld[0], 0, B, n, d->kp[0], 1, HOBC_TC_OUT_F32, out, nullptr, nullptr, n, 0);
    }
    const int n0 = d->n[0], n1 = d->n[1];
    hobc_status s = hobc_tc_split(gf, n1, (long long)n0 * n1, n0, n1, d->w_hi[0] + z0 * d->w_bs[0],
                                  d->w_lo[0] + z0 * d->w_bs[0], d->w_ld[0], d->w_bs[0], n0, B, p->stream);
    if (s != HOBC_OK) return s;
    ++p->launches;
    // rows: R[t1][r] = sum_j T1^{-1}[t1][j] g[r][j], computed as C[r][t1] and stored transposed
    s = gemm(p, d->w_hi[0] + z0 * d->w_bs[0], d->w_lo[0] + z0 * d->w_bs[0], d->w_ld[0], d->w_bs[0], d->m_hi[0],
             d->m_lo[0], d->m_ld[0], 0, n0, n1, d->kp[1], B, HOBC_TC_OUT_SPLIT_T, nullptr,
             d->w_hi[1] + z0 * d->w_bs[1], d->w_lo[1] + z0 * d->w_bs[1], d->w_ld[1], d->w_bs[1]);
    if (s != HOBC_OK) return s;
    // columns: ghat[t1][t0] = sum_r T0^{-1}[t0][r] R[t1][r], computed as C[t0][t1] and stored transposed
    return gemm(p, d->m_hi[1], d->m_lo[1], d->m_ld[1], 0, d->w_hi[1] + z0 * d->w_bs[1], d->w_lo[1] + z0 * d->w_bs[1],
                d->w_ld[1], d->w_bs[1], n0, n1, d->kp[0], B, HOBC_TC_OUT_F32_T, out, nullptr, nullptr, n0,
                (long long)n0 * n1);
}

// Fourier family: filter (complex) + split, then the synthesis products.
static hobc_status dense_filter_synthesis_fourier(hobc_plan_s* p, const float2* spec, const FilterDesc& fd,
                                                  float* f) {
    hobc_dense_s* d = p->dense;
    const int B = p->desc.batch;
    const size_t z0 = p->item0;
    const int W = d->W;
    if (d->nax == 1) {
        const int n = d->n[0];
        tc::k_filter_split_cplx<<<1024, 256, 0, p->stream>>>(spec, (long long)p->spec_elems, 1, W, 1, axis0(p), fd, B,
                                                              d->w_hi[2] + z0 * d->w_ld[2], d->w_lo[2] + z0 * d->w_ld[2],
                                                              d->w_ld[2], 0);
        hobc_status s = check("k_filter_split_cplx");
        if (s != HOBC_OK) return s;
        ++p->launches;
        return gemm(p, d->w_hi[2] + z0 * d->w_ld[2], d->w_lo[2] + z0 * d->w_ld[2], d->w_ld[2], 0, d->m_hi[2],
                    d->m_lo[2], d->m_ld[2], 0, B, n, d->k2, 1, HOBC_TC_OUT_F32, f, nullptr, nullptr, n, 0);
    }
    const int n0 = d->n[0], n1 = d->n[1];
    tc::k_filter_split_cplx<<<1024, 256, 0, p->stream>>>(spec, (long long)p->spec_elems, W, n0, 2, axis0(p), fd, B,
                                                          d->w_hi[2] + z0 * d->w_bs[2], d->w_lo[2] + z0 * d->w_bs[2],
                                                          d->w_ld[2], d->w_bs[2]);
    hobc_status s = check("k_filter_split_cplx");
    if (s != HOBC_OK) return s;
    ++p->launches;
    // columns: Y[2r + p][c] = sum_(t0, q) M0s[2r + p][(t0, q)] X[c][(t0, q)]
    s = gemm(p, d->m_hi[2], d->m_lo[2], d->m_ld[2], 0, d->w_hi[2] + z0 * d->w_bs[2], d->w_lo[2] + z0 * d->w_bs[2],
             d->w_ld[2], d->w_bs[2], 2 * n0, W, d->k2, B, HOBC_TC_OUT_SPLIT, nullptr, d->w_hi[3] + z0 * d->w_bs[3],
             d->w_lo[3] + z0 * d->w_bs[3], d->kw, d->w_bs[3]);
    if (s != HOBC_OK) return s;
    // rows: f[r][j] = sum_(q, c) M1s[j][(q, c)] Y(r)[(q, c)], computed as C[j][r] and stored transposed
    return gemm(p, d->m_hi[3], d->m_lo[3], d->m_ld[3], 0, d->w_hi[3] + z0 * d->w_bs[3], d->w_lo[3] + z0 * d->w_bs[3],
                d->w_ld[3], d->w_bs[3], n1, n0, 2 * d->kw, B, HOBC_TC_OUT_F32_T, f, nullptr, nullptr, n1,
                (long long)n0 * n1);
}

hobc_status dense_filter_synthesis(hobc_plan_s* p, const void* ghat, const void* D, const int* mu_idx,
                                   const double* mu_val, void* f) {
    hobc_dense_s* d = p->dense;
    const int B = p->desc.batch;
    const size_t z0 = p->item0;
    const FilterDesc fd = filter_desc(p, D, mu_idx, mu_val);
    if (d->fourier)
        return dense_filter_synthesis_fourier(p, static_cast<const float2*>(ghat), fd, static_cast<float*>(f));
    const int rows = d->nax == 2 ? d->n[1] : 1, cols = d->nax == 2 ? d->n[0] : d->n[0];
    __nv_bfloat16* xh = d->w_hi[2] + z0 * (d->nax == 2 ? d->w_bs[2] : d->w_ld[2]);
    __nv_bfloat16* xl = d->w_lo[2] + z0 * (d->nax == 2 ? d->w_bs[2] : d->w_ld[2]);
    tc::k_filter_split<<<1024, 256, 0, p->stream>>>(static_cast<const float*>(ghat), (long long)p->spec_elems, rows,
                                                     cols, d->nax, axis0(p), fd, B, xh, xl, d->w_ld[2], d->w_bs[2]);
    hobc_status s = check("k_filter_split");
    if (s != HOBC_OK) return s;
    ++p->launches;
    return dense_synthesis_from_x(p, static_cast<float*>(f));
}

hobc_status dense_synthesis(hobc_plan_s* p, const void* c, void* y) {
    return dense_filter_synthesis(p, c, nullptr, nullptr, nullptr, y);
}

}  // namespace hobc


extern "C" {

int hobc_tc_tile_m(void) { return tc::BM; }
int hobc_tc_tile_n(void) { return tc::BN; }
int hobc_tc_tile_k(void) { return tc::BK; }

hobc_status hobc_tc_split(const float* src, long long src_ld, long long src_batch_stride, int rows, int cols,
                          void* hi, void* lo, long long ld, long long batch_stride, int rows_padded, int batch,
                          void* cuda_stream) {
    if (!src || !hi || !lo || rows < 0 || cols < 0 || batch < 1 || rows_padded < rows || ld < cols) return HOBC_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    tc::k_split<<<1024, 256, 0, st>>>(src, src_ld, src_batch_stride, rows, cols, static_cast<__nv_bfloat16*>(hi),
                                      static_cast<__nv_bfloat16*>(lo), ld, batch_stride, rows_padded, batch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error("hobc_tc_split", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

hobc_status hobc_tc_gemm(const hobc_tc_operand* a, const hobc_tc_operand* b, int m, int n, int k, int batch,
                         const hobc_tc_output* out, int* err_dev, void* cuda_stream) {
    if (!a || !b || !out || !err_dev || m < 1 || n < 1 || k < 1 || batch < 1 || batch > 65535) return HOBC_ERR_ARG;
    if (!a->hi || !a->lo || !b->hi || !b->lo) return HOBC_ERR_ARG;
    if (a->ld % 8 || b->ld % 8 || a->ld < k || b->ld < k) return HOBC_ERR_ARG;     // 16-byte rows
    if (k % tc::BK) return HOBC_ERR_ARG;                                             // padded K
    if (a->batch_stride % a->ld || b->batch_stride % b->ld) return HOBC_ERR_ARG;     // whole rows per problem
    if (out->mode < HOBC_TC_OUT_F32 || out->mode > HOBC_TC_OUT_SPLIT_T) return HOBC_ERR_ARG;
    const bool split = out->mode == HOBC_TC_OUT_SPLIT || out->mode == HOBC_TC_OUT_SPLIT_T;
    if (split ? (!out->hi || !out->lo) : !out->f32) return HOBC_ERR_ARG;
    const long long mp = (m + tc::BM - 1) / tc::BM * tc::BM, np = (n + tc::BN - 1) / tc::BN * tc::BN;
    const long long a_rpp = a->batch_stride / a->ld, b_rpp = b->batch_stride / b->ld;
    if ((a_rpp && a_rpp < mp) || (b_rpp && b_rpp < np)) return HOBC_ERR_ARG;     // padded rows per problem
    if (a_rpp * (batch - 1) + mp > INT32_MAX || b_rpp * (batch - 1) + np > INT32_MAX) return HOBC_ERR_SIZE;
    hobc_status s = tc::encode_maps();
    if (s != HOBC_OK) return s;
    tc::Maps maps;
    s = tc::make_map(&maps.a_hi, a->hi, k, a->ld, a_rpp * (batch - 1) + mp, tc::BM);
    if (s == HOBC_OK) s = tc::make_map(&maps.a_lo, a->lo, k, a->ld, a_rpp * (batch - 1) + mp, tc::BM);
    if (s == HOBC_OK) s = tc::make_map(&maps.b_hi, b->hi, k, b->ld, b_rpp * (batch - 1) + np, tc::BN);
    if (s == HOBC_OK) s = tc::make_map(&maps.b_lo, b->lo, k, b->ld, b_rpp * (batch - 1) + np, tc::BN);
    if (s != HOBC_OK) return s;
    cudaError_t e = cudaFuncSetAttribute(tc::k_gemm_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc::SMEM_BYTES);
    if (e != cudaSuccess) { set_last_error("hobc_tc_gemm", e); return HOBC_ERR_CUDA; }
    tc::Output O{out->mode, out->f32, static_cast<__nv_bfloat16*>(out->hi), static_cast<__nv_bfloat16*>(out->lo),
                 out->ld, out->batch_stride, out->rows, out->cols};
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    const int ntn = (int)(np / tc::BN), ntm = (int)(mp / tc::BM);
    const long long ntiles = (long long)ntn * ntm * batch;
    if (ntiles > INT32_MAX) return HOBC_ERR_SIZE;
    const unsigned grid = (unsigned)std::min<long long>(ntiles, sms);
    tc::k_gemm_split<<<grid, tc::THREADS, tc::SMEM_BYTES, reinterpret_cast<cudaStream_t>(cuda_stream)>>>(
        maps, (int)a_rpp, (int)b_rpp, k / tc::BK, ntn, ntm, (int)ntiles, O, err_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error("hobc_tc_gemm", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

hobc_status hobc_plan_status(hobc_plan* p) {
    if (!p) return HOBC_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) { set_last_error("hobc_plan_status", e); return HOBC_ERR_CUDA; }
    if (!p->dense) return HOBC_OK;
    int flag = 0;
    e = cudaMemcpy(&flag, p->dense->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flag) e = cudaMemset(p->dense->err, 0, sizeof(int));
    if (e != cudaSuccess) { set_last_error("hobc_plan_status", e); return HOBC_ERR_CUDA; }
    if (flag) {
        set_last_error_text("a tensor-core pipeline wait gave up; the affected tiles were not written");
        return HOBC_ERR_TIMEOUT;
    }
    return HOBC_OK;
}

}  // extern "C"
