// Internal declarations of the surrogate MLP kernels.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

namespace pcmd {

// GEMM epilogues: D = A[M,K] . B[N,K]^T accumulated in FP32 (TMEM), then
enum GemmEpilogue : int {
    kEpiF32 = 0,           // C (FP32) = D
    kEpiBiasF32 = 1,       // C (FP32) = D + bias[n]
    kEpiBiasGeluBf16 = 2,  // C (BF16) = gelu(D + bias[n]);  aux (BF16) = D + bias[n]
    kEpiBiasBf16 = 3,      // C (BF16) = D + bias[n]
};

struct GemmArgs {
    void *c;          // output, row-major [M][ldc]
    void *aux;        // pre-activation output (kEpiBiasGeluBf16), row-major [M][ldc]
    const float *bias;
    int m, n, k, ldc;
    uint32_t *err;
};

// Launch C = A . B^T (both operands K-major BF16, row strides lda / ldb elements, multiples
// of 8).  Builds the TMA descriptors on the host.
cudaError_t launch_gemm_bf16(const void *a, int lda, const void *b, int ldb, const GemmArgs &g,
                             int epilogue, cudaStream_t st);

}  // namespace pcmd
