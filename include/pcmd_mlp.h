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
 * epilogue; NULL: the pre-activations are not stored).  d_err: device uint32 error word (bit 2 set if a bounded wait ran out), may not be
 * NULL.  Asynchronous. */
pcmd_status pcmd_gemm_bf16(const void *d_a, int lda, const void *d_b, int ldb, void *d_c, int ldc,
                           const float *d_bias, void *d_aux, int m, int n, int k, int epilogue,
                           uint32_t *d_err, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* The surrogate network: an MLP dims[0] -> dims[1] -> ... -> dims[n_layers] with GELU on the */
/* hidden layers and a linear FP32 output, BF16 weights and activations, FP32 master weights  */
/* and Adam.  Inputs are the raw model parameters, normalised in a kernel to [-1, 1] over the */
/* box [in_lo, in_hi]; targets are ln(1 + m) of Hess counts m.                                 */
/* ---------------------------------------------------------------------------------------- */
typedef struct pcmd_mlp pcmd_mlp;

/* Create a network on the current device.  h_dims [n_layers + 1]: multiples of 8, dims[0] <= 64
 * is the padded input width; n_in <= dims[0] raw inputs with box h_in_lo / h_in_hi [n_in];
 * max_batch a multiple of 8.  Weights: LeCun-normal from a Mersenne twister seeded with `seed`,
 * biases zero.  All work runs on `stream`.  *out is NULL on error. */
pcmd_status pcmd_mlp_create(const int *h_dims, int n_layers, int n_in, const float *h_in_lo,
                            const float *h_in_hi, int max_batch, uint64_t seed, void *stream,
                            pcmd_mlp **out);
void pcmd_mlp_destroy(pcmd_mlp *mlp);
const char *pcmd_mlp_last_error(const pcmd_mlp *mlp);

/* Forward pass of B rows (B a multiple of 8, <= max_batch): theta [B][n_in] FP32, on the device
 * when on_device != 0 else on the host; d_out [B][dims[n_layers]] FP32 (may be NULL: the output
 * stays inside the network, see pcmd_mlp_output).  Asynchronous. */
pcmd_status pcmd_mlp_forward(pcmd_mlp *mlp, const float *theta, int on_device, int B, float *d_out);

/* Device pointer of the last forward output [B][dims[n_layers]] FP32 (owned by the network). */
const float *pcmd_mlp_output(const pcmd_mlp *mlp);

/* Output and loss convention: 0 (default) = the output is ln(1 + m) trained with the squared
 * error; 1 = the output is the log expected count trained with the Poisson deviance
 * exp(yhat) - m yhat on the counts m (the form the Poisson likelihood needs). */
pcmd_status pcmd_mlp_set_loss(pcmd_mlp *mlp, int poisson);

/* Training targets of the next step from the Hess counts d_hess [B][dims[n_layers]] (uint32,
 * device): ln(1 + m), or m itself under the Poisson convention; or given FP32 targets d_y.
 * Asynchronous. */
pcmd_status pcmd_mlp_targets(pcmd_mlp *mlp, const uint32_t *d_hess, int B);
pcmd_status pcmd_mlp_set_targets(pcmd_mlp *mlp, const float *d_y, int B);

/* One step: forward on theta (as in pcmd_mlp_forward), loss (sum (yhat - y)^2 / 2, or the Poisson
 * deviance) / B, backward
 * through every layer with tensor-core GEMMs, and (update != 0) an Adam step with learning rate
 * lr (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  Asynchronous. */
pcmd_status pcmd_mlp_train_step(pcmd_mlp *mlp, const float *theta, int on_device, int B, float lr,
                                int update);

/* Loss of the last step (host); synchronises and reports a latched GEMM error. */
pcmd_status pcmd_mlp_loss(pcmd_mlp *mlp, double *h_loss);

/* Poisson log-likelihood (the alternative of Section 2.5) of the last forward pass's B
 * predicted diagrams against data counts d_data_hess [dims[n_layers]] (device): predicted counts
 * of the network's image (exp(yhat), or expm1(yhat) under the squared-error convention) times
 * `scale` (model pixels / network-image pixels), floored at 1/2, times `ratio` (data pixels /
 * model pixels); sum d ln mh - mh - ln Gamma(d + 1).  Per-bin terms in FP32, sums in FP64 (the
 * data term in FP64 throughout).  scale and ratio must be positive (PCMD_ERR_ARG).  h_ll [B];
 * synchronises. */
pcmd_status pcmd_mlp_loglike(pcmd_mlp *mlp, int B, const uint32_t *d_data_hess, double scale,
                             double ratio, double *h_ll);

/* Forward pass and surrogate log-likelihood in one call: the output layer's epilogue forms
 * the per-bin terms of pcmd_mlp_loglike straight from the tensor-memory accumulator (one
 * partial sum per row and 64-column block, added in a fixed order), so the B x dims[n_layers]
 * predicted diagrams are never written to memory.  Arguments as pcmd_mlp_forward and
 * pcmd_mlp_loglike; d_data_hess 16-byte aligned; B a multiple of 8.  pcmd_mlp_output is left
 * unchanged.  Synchronises; PCMD_ERR_TIMEOUT if a bounded wait inside a GEMM ran out. */
pcmd_status pcmd_mlp_forward_loglike(pcmd_mlp *mlp, const float *theta, int on_device, int B,
                                     const uint32_t *d_data_hess, double scale, double ratio,
                                     double *h_ll);

/* Host copies of layer l's FP32 weights [dims[l+1]][dims[l]], bias, and the last step's gradients
 * (any pointer may be NULL); set_layer replaces weights and bias.  Synchronous. */
pcmd_status pcmd_mlp_get_layer(pcmd_mlp *mlp, int l, float *h_w, float *h_b, float *h_gw, float *h_gb);
pcmd_status pcmd_mlp_set_layer(pcmd_mlp *mlp, int l, const float *h_w, const float *h_b);

#ifdef __cplusplus
}
#endif
#endif /* PCMD_MLP_H */
