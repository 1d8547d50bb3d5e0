/*
 * pcmd_mlp.h -- C ABI of the surrogate network kernels (BF16 tensor-core GEMM, MLP training and
 * inference).  The paper has no surrogate: this is the learned emulator that maps the model
 * parameters (Table 1) to the log Hess diagram of Section 2.5 so that a sampler can pre-screen
 * proposals; the exact simulator (pcmd.h) stays the judge of every accepted point.
 *
 * Conventions as in pcmd.h: device pointers d_, host pointers h_, status codes, asynchronous on
 * the given stream unless stated otherwise, nothing allocated on behalf of the caller except
 * inside a pcmd_mlp object.
 */
#ifndef PCMD_MLP_H
#define PCMD_MLP_H

#include <stddef.h>
#include <stdint.h>

#include "pcmd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* GEMM epilogues */
enum {
    PCMD_GEMM_F32 = 0,            /* C (FP32) = A . B^T */
    PCMD_GEMM_BIAS_F32 = 1,       /* C (FP32) = A . B^T + bias */
    PCMD_GEMM_BIAS_GELU_BF16 = 2, /* C (BF16) = gelu(A . B^T + bias); aux (BF16) = A . B^T + bias */
    PCMD_GEMM_BIAS_BF16 = 3       /* C (BF16) = A . B^T + bias */
};

/* C[m][n] = epilogue(sum_k A[m][k] B[n][k]) with BF16 A (row-major, row stride lda elements)
 * and BF16 B (row-major [n][k], row stride ldb), FP32 accumulation on the tensor cores
 * (tcgen05.mma, operands staged by TMA).  lda, ldb: multiples of 8, >= k; A and B 16-byte
 * aligned; C row stride ldc elements; bias [n] FP32 (bias epilogues); aux like C (GELU
 * epilogue).  d_err: device uint32 error word (bit 2 set if a bounded wait ran out), may not be
 * NULL.  Asynchronous. */
pcmd_status pcmd_gemm_bf16(const void *d_a, int lda, const void *d_b, int ldb, void *d_c, int ldc,
                           const float *d_bias, void *d_aux, int m, int n, int k, int epilogue,
                           uint32_t *d_err, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PCMD_MLP_H */
