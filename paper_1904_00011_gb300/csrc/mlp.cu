// C ABI of the surrogate network kernels (include/pcmd_mlp.h).
#include "../../include/pcmd_mlp.h"
#include "mlp_internal.h"

using namespace pcmd;

extern "C" pcmd_status pcmd_gemm_bf16(const void *d_a, int lda, const void *d_b, int ldb, void *d_c,
                                      int ldc, const float *d_bias, void *d_aux, int m, int n, int k,
                                      int epilogue, uint32_t *d_err, void *stream) {
    if (!d_a || !d_b || !d_c || !d_err || m <= 0 || n <= 0 || k <= 0 || ldc < n) return PCMD_ERR_ARG;
    if ((epilogue == PCMD_GEMM_BIAS_F32 || epilogue == PCMD_GEMM_BIAS_GELU_BF16 ||
         epilogue == PCMD_GEMM_BIAS_BF16) && !d_bias)
        return PCMD_ERR_ARG;
    if (epilogue == PCMD_GEMM_BIAS_GELU_BF16 && !d_aux) return PCMD_ERR_ARG;
    if (epilogue < 0 || epilogue > 3) return PCMD_ERR_ARG;
    GemmArgs g;
    g.c = d_c;
    g.aux = d_aux;
    g.bias = d_bias;
    g.m = m;
    g.n = n;
    g.k = k;
    g.ldc = ldc;
    g.err = d_err;
    cudaError_t e = launch_gemm_bf16(d_a, lda, d_b, ldb, g, epilogue, (cudaStream_t)stream);
    if (e == cudaErrorInvalidValue) return PCMD_ERR_ARG;
    return e == cudaSuccess ? PCMD_OK : PCMD_ERR_CUDA;
}
