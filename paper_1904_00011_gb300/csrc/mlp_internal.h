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
    kEpiPoissonLL = 4,     // no C: per (row, 64-column block) sums of the surrogate likelihood terms
};

// Output tiles are 128 x kGemmTileN; the likelihood epilogue leaves kGemmLlBlocks partial sums
// per row and tile (one per epilogue warp's column block).
constexpr int kGemmTileN = 256;
constexpr int kGemmLlBlocks = 4;

struct GemmArgs {                 // every field has a default: an unset pointer is null
    void *c = nullptr;            // output, row-major [M][ldc]
    void *aux = nullptr;          // pre-activation output (kEpiBiasGeluBf16), or null: not stored
    const float *bias = nullptr;
    int m = 0, n = 0, k = 0, ldc = 0;
    uint32_t *err = nullptr;
    int tma_store = 0;   // set by the launcher: outputs go through TMA stores
    // kEpiPoissonLL: data counts [n], the term of each bin (y = D + bias) as in the surrogate
    // likelihood, partial sums to ll_part[row * ll_ld + 64-column block index]
    const uint32_t *ll_data = nullptr;
    double *ll_part = nullptr;
    int ll_ld = 0, ll_poisson = 1;
    float ll_sc = 1.0f, ll_lsc = 0.0f, ll_ra = 1.0f, ll_lra = 0.0f;
};

// One bin of the surrogate Poisson likelihood: the log-rate mode reads y as ln(rate), so
// ln mh = max(y + ln scale, ln 1/2) + ln ratio needs no logarithm; the other mode reads y as
// ln(1 + rate).  mh = max(rate * scale, 1/2) * ratio; the term is d ln mh - mh.
__device__ __forceinline__ float surrogate_ll_term(float y, uint32_t d, float sc, float lsc, float ra,
                                                   float lra, int poisson) {
    float mh, lmh;
    if (poisson) {
        mh = fmaxf(__expf(y) * sc, 0.5f) * ra;
        lmh = fmaxf(y + lsc, -0.69314718f) + lra;
    } else {
        mh = fmaxf(expm1f(y) * sc, 0.5f) * ra;
        lmh = logf(mh);
    }
    return (float)d * lmh - mh;
}

// Launch C = A . B^T (both operands K-major BF16, row strides lda / ldb elements, multiples
// of 8).  Builds the TMA descriptors on the host.
cudaError_t launch_gemm_bf16(const void *a, int lda, const void *b, int ldb, const GemmArgs &g,
                             int epilogue, cudaStream_t st);

}  // namespace pcmd
