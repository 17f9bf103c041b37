// Dense transforms on the 5th-generation tensor cores (split-BF16).
//
// Every pass of the dense mode is C[M x N] = A[M x K] . B[N x K]^T with both
// operands K-major in HBM and each operand held as a pair of bfloat16 arrays
// (hi = bf16(x), lo = bf16(x - hi)); the three products hi.hi + hi.lo + lo.hi
// accumulate in FP32 in tensor memory, which keeps about 16 significant bits
// of every product.  One CTA (four warps) computes a 128 x 256 tile: all
// threads stage K-slices of 64 into shared memory with cp.async in the
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix), one
// thread issues tcgen05.mma and commits to an mbarrier per stage, and the
// four warps read their 32 accumulator lanes back with tcgen05.ld for the
// epilogue.  Every mbarrier wait is bounded; a wait that gives up sets an
// error word that the host reads.
#include <cuda_bf16.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/hobc_tc.h"
#include "hobc_internal.h"

namespace hobc {
namespace tc {

constexpr int BM = 128;          // tile rows (accumulator lanes)
constexpr int BN = 256;          // tile columns (accumulator columns)
constexpr int BK = 64;           // K per stage (eight 16-byte core-matrix columns)
constexpr int STAGES = 2;
constexpr int THREADS = 128;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;     // A hi, A lo, B hi, B lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;    // + barriers and the TMEM slot
constexpr unsigned WAIT_LIMIT = 1u << 22;                  // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle: start address, the byte
// distance between core matrices adjacent in K (leading) and in M/N (stride).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lead, uint32_t stride) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lead >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((stride >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;     // descriptor version of this architecture family
    return d;                    // base offset 0, swizzle none
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

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}

// Rows [0, R) x K-slice [k0, k0 + 64) of a K-major bf16 matrix (leading
// dimension ld elements) into the core-matrix layout: row r, 16-byte column c
// at ((r / 8) * 8 + c) * 128 + (r % 8) * 16.  Thread i copies the i-th 16 bytes
// of that layout, so a warp's shared-memory stores are contiguous and its
// global reads are 64 contiguous bytes from each of 8 rows.
template <int R>
__device__ __forceinline__ void stage_tile(uint32_t sbase, const __nv_bfloat16* __restrict__ g, long long ld,
                                           int k0) {
#pragma unroll 4
    for (int i = threadIdx.x; i < R * 8; i += THREADS) {
        const int grp = i >> 6, c = (i >> 3) & 7, rr = i & 7;
        cp_async16(sbase + (uint32_t)(i << 4), g + (long long)(grp * 8 + rr) * ld + k0 + c * 8);
    }
}

struct Operand {                 // one split operand: hi and lo arrays, K-major
    const __nv_bfloat16* hi;
    const __nv_bfloat16* lo;
    long long ld;                // elements between rows
    long long batch_stride;      // elements between problems (0: shared)
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

// C tile (blockIdx.x: N tile, blockIdx.y: M tile, blockIdx.z: problem).
__global__ void __launch_bounds__(THREADS, 1)
k_gemm_split(Operand A, Operand B, int KT, Output out, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + STAGES * STAGE_BYTES + 64);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const long long z = blockIdx.z;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const __nv_bfloat16* Ahi = A.hi + z * A.batch_stride + (long long)m0 * A.ld;
    const __nv_bfloat16* Alo = A.lo + z * A.batch_stride + (long long)m0 * A.ld;
    const __nv_bfloat16* Bhi = B.hi + z * B.batch_stride + (long long)n0 * B.ld;
    const __nv_bfloat16* Blo = B.lo + z * B.batch_stride + (long long)n0 * B.ld;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[s])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("fence.proxy.async.shared::cta;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = instr_desc(BM, BN);
    bool ok = true;

    for (int kt = 0; kt < KT; ++kt) {
        const int s = kt % STAGES;
        unsigned char* st = smem + s * STAGE_BYTES;
        if (kt >= STAGES) {      // the MMAs of tile kt - STAGES read this stage
            if (!wait_bounded(&bars[s], (uint32_t)((kt / STAGES - 1) & 1))) ok = false;
        }
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        const uint32_t sa = smem_u32(st);
        stage_tile<BM>(sa, Ahi, A.ld, kt * BK);
        stage_tile<BM>(sa + A_BYTES, Alo, A.ld, kt * BK);
        stage_tile<BN>(sa + 2 * A_BYTES, Bhi, B.ld, kt * BK);
        stage_tile<BN>(sa + 2 * A_BYTES + B_BYTES, Blo, B.ld, kt * BK);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a_hi = sa, a_lo = sa + A_BYTES, b_hi = sa + 2 * A_BYTES, b_lo = b_hi + B_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint32_t ko = kk * 256;     // two core matrices of K per MMA
                const uint64_t dah = smem_desc(a_hi + ko, 128, 1024), dal = smem_desc(a_lo + ko, 128, 1024);
                const uint64_t dbh = smem_desc(b_hi + ko, 128, 1024), dbl = smem_desc(b_lo + ko, 128, 1024);
                mma(tmem, dah, dbh, idesc, (kt | kk) ? 1u : 0u);
                mma(tmem, dah, dbl, idesc, 1u);
                mma(tmem, dal, dbh, idesc, 1u);
            }
            commit(&bars[s]);
        }
        __syncthreads();
    }
    // all MMAs issued so far complete in order: wait for the last commit
    if (ok && KT > 0) {
        const int last = KT - 1;
        if (!wait_bounded(&bars[last % STAGES], (uint32_t)((last / STAGES) & 1))) ok = false;
    }
    if (!ok && lane == 0) atomicOr(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (ok) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(lane_base + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < out.rows) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col >= out.cols) break;
                    const float v = __uint_as_float(r[j]);
                    if (out.mode == HOBC_TC_OUT_F32) {
                        out.f32[z * out.batch_stride + (long long)row * out.ld + col] = v;
                    } else if (out.mode == HOBC_TC_OUT_F32_T) {
                        out.f32[z * out.batch_stride + (long long)col * out.ld + row] = v;
                    } else if (out.mode == HOBC_TC_OUT_SPLIT) {
                        split_store(out.hi, out.lo, z * out.batch_stride + (long long)row * out.ld + col, v);
                    } else {
                        split_store(out.hi, out.lo, z * out.batch_stride + (long long)col * out.ld + row, v);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
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

}  // namespace tc
}  // namespace hobc

using namespace hobc;

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
    if (out->mode < HOBC_TC_OUT_F32 || out->mode > HOBC_TC_OUT_SPLIT_T) return HOBC_ERR_ARG;
    const bool split = out->mode == HOBC_TC_OUT_SPLIT || out->mode == HOBC_TC_OUT_SPLIT_T;
    if (split ? (!out->hi || !out->lo) : !out->f32) return HOBC_ERR_ARG;
    cudaError_t e = cudaFuncSetAttribute(tc::k_gemm_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc::SMEM_BYTES);
    if (e != cudaSuccess) { set_last_error("hobc_tc_gemm", e); return HOBC_ERR_CUDA; }
    tc::Operand A{static_cast<const __nv_bfloat16*>(a->hi), static_cast<const __nv_bfloat16*>(a->lo), a->ld,
                  a->batch_stride};
    tc::Operand B{static_cast<const __nv_bfloat16*>(b->hi), static_cast<const __nv_bfloat16*>(b->lo), b->ld,
                  b->batch_stride};
    tc::Output O{out->mode, out->f32, static_cast<__nv_bfloat16*>(out->hi), static_cast<__nv_bfloat16*>(out->lo),
                 out->ld, out->batch_stride, out->rows, out->cols};
    dim3 grid((unsigned)((n + tc::BN - 1) / tc::BN), (unsigned)((m + tc::BM - 1) / tc::BM), (unsigned)batch);
    tc::k_gemm_split<<<grid, tc::THREADS, tc::SMEM_BYTES, reinterpret_cast<cudaStream_t>(cuda_stream)>>>(
        A, B, k / tc::BK, O, err_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error("hobc_tc_gemm", e); return HOBC_ERR_CUDA; }
    return HOBC_OK;
}

}  // extern "C"
