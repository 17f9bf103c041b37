/*
 * Dense transform engine on the tensor cores (split-BF16).  The paper computes
 * T_X^{-1} g and T_X c with fast trigonometric transforms (Sec. 3, Sec. 6);
 * for real families any of these products is also a dense matrix product,
 * C = A . B^T, which this engine runs on tcgen05 tensor cores with every
 * operand split into two bfloat16 arrays (hi = bf16(x), lo = bf16(x - hi))
 * and the three products hi.hi + hi.lo + lo.hi accumulated in FP32.  The
 * result keeps about 16 significant bits of each product: per entry
 * |C - A.B^T| <= (2^-14 + K 2^-24) (|A| |B|^T).  The Fourier family's T_F is
 * complex (Eq. (eq:Tf)); its products run as real products on (re, im) pairs:
 * the row analysis against the (Re, Im) rows of T_1^{-1} on the stored half
 * spectrum, the column analysis and synthesis against the real 2 x 2 block form
 * of T_0^{-1} and T_0, and the row synthesis against the FP64 path's response
 * to a unit real or imaginary entry of the half spectrum.
 *
 * Conventions are those of hobc.h: device pointers, asynchronous on the given
 * stream, errors as hobc_status with hobc_last_error() for CUDA failures.
 */
#ifndef HOBC_TC_H
#define HOBC_TC_H

#include "hobc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Output layouts of hobc_tc_gemm. */
enum {
    HOBC_TC_OUT_F32 = 0,       /* f32[z][m][n] at z*batch_stride + m*ld + n            */
    HOBC_TC_OUT_F32_T = 1,     /* f32[z][n][m] at z*batch_stride + n*ld + m            */
    HOBC_TC_OUT_SPLIT = 2,     /* hi/lo bf16 at z*batch_stride + m*ld + n              */
    HOBC_TC_OUT_SPLIT_T = 3    /* hi/lo bf16 at z*batch_stride + n*ld + m              */
};

typedef struct {
    const void* hi;            /* bf16, row r of problem z at z*batch_stride + r*ld    */
    const void* lo;            /* bf16, same layout                                    */
    long long ld;              /* elements between rows: a multiple of 8, >= K         */
    long long batch_stride;    /* elements between problems (0: one matrix for all)    */
} hobc_tc_operand;

typedef struct {
    int mode;                  /* HOBC_TC_OUT_*                                        */
    float* f32;                /* FP32 modes                                           */
    void* hi;                  /* split modes: bf16 hi / lo arrays                     */
    void* lo;
    long long ld;
    long long batch_stride;
    int rows;                  /* entries with m >= rows or n >= cols are not written  */
    int cols;
} hobc_tc_output;

/* Tile sizes: A must hold rows [0, ceil(m / tile_m) * tile_m) and B rows
 * [0, ceil(n / tile_n) * tile_n) of every problem (zero padding), K a multiple
 * of tile_k (the padded columns zero). */
int hobc_tc_tile_m(void);
int hobc_tc_tile_n(void);
int hobc_tc_tile_k(void);

/* C[z] = A[z] . B[z]^T for z < batch (batch <= 65535); m, n the valid extent
 * of C, k the padded K.  err_dev: an int the kernel ORs 1 into if a bounded
 * wait on its tensor-core pipeline gave up (the tile is then not written). */
hobc_status hobc_tc_gemm(const hobc_tc_operand* a, const hobc_tc_operand* b, int m, int n, int k, int batch,
                         const hobc_tc_output* out, int* err_dev, void* cuda_stream);

/* Split FP32 [batch][rows][cols] (row stride src_ld, problem stride
 * src_batch_stride) into zero-padded bf16 hi/lo [batch][rows_padded][ld]. */
hobc_status hobc_tc_split(const float* src, long long src_ld, long long src_batch_stride, int rows, int cols,
                          void* hi, void* lo, long long ld, long long batch_stride, int rows_padded, int batch,
                          void* cuda_stream);

/* Synchronise the plan's stream and report whether a bounded tensor-core wait
 * of an HOBC_SPLIT_BF16 plan gave up since the last call (HOBC_ERR_TIMEOUT,
 * flag cleared); HOBC_OK otherwise and for other precisions. */
hobc_status hobc_plan_status(hobc_plan* plan);

#ifdef __cplusplus
}
#endif

#endif /* HOBC_TC_H */
