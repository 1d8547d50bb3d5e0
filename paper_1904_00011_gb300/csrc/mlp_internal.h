// Internal declarations of the surrogate MLP kernels.
#pragma once
#include <stdint.h>
#include <cmath>
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

// Constants of the surrogate likelihood of one call: model counts = rate * scale, floored at
// 1/2, times ratio = N_d / N_m.
struct LLConsts {
    float c1, c0;      // ln(scale * ratio), ln(1/2) + ln(ratio)
    float sc, ra;      // scale, ratio (the ln(1 + m) convention)
};

__host__ inline LLConsts ll_consts(double scale, double ratio) {
    LLConsts k;
    k.c1 = (float)(std::log(scale) + std::log(ratio));
    k.c0 = (float)(std::log(0.5) + std::log(ratio));
    k.sc = (float)scale;
    k.ra = (float)ratio;
    return k;
}

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
    LLConsts llk = {0.0f, -0.69314718f, 1.0f, 1.0f};
};


// One bin of the surrogate Poisson likelihood, d ln mh - mh.  The log-rate output y gives
// ln mh = u = max(y + ln scale, ln 1/2) + ln ratio and mh = e^u (no logarithm); the ln(1 + m)
// output gives mh = max(expm1(y) scale, 1/2) ratio.
__device__ __forceinline__ float surrogate_ll_term(float y, uint32_t d, const LLConsts &k, int poisson) {
    if (poisson) {
        const float u = fmaxf(y + k.c1, k.c0);
        return fmaf((float)d, u, -__expf(u));
    }
    const float mh = fmaxf(expm1f(y) * k.sc, 0.5f) * k.ra;
    return (float)d * logf(mh) - mh;
}

// Launch C = A . B^T (both operands K-major BF16, row strides lda / ldb elements, multiples
// of 8).  Builds the TMA descriptors on the host.
cudaError_t launch_gemm_bf16(const void *a, int lda, const void *b, int ldb, const GemmArgs &g,
                             int epilogue, cudaStream_t st);

}  // namespace pcmd
