// The surrogate network (include/pcmd_mlp.h): an MLP from the model parameters (Table 1) to the
// log Hess diagram ln(1 + m) of Section 2.5, trained with its own kernels: tcgen05 BF16 GEMMs
// (mlp_gemm.cu) for every product, FP32 master weights and Adam, BF16 activations.
//
// Layer l maps X_l [B][K_l] to Z_l = X_l W_l^T + b_l; hidden layers apply GELU (exact, erf form),
// the last layer is linear in FP32.  Loss: L = sum (yhat - y)^2 / (2B).  Backward per layer:
// dZ = dA * gelu'(Z) (hidden), dW = dZ^T X, db = column sums of dZ, dX = dZ W.  Both GEMM
// operands are K-major, so the kernels below also write the transposes dZ^T and X^T, and Adam
// writes W in both layouts.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/pcmd_mlp.h"
#include "mlp_internal.h"

using namespace pcmd;

namespace {

constexpr int kTT = 32;   // transpose tile

__device__ __forceinline__ float gelu_grad(float z) {
    const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
    return cdf + z * pdf;
}

// Normalised inputs: x = 2 (theta - lo) / (hi - lo) - 1 for the first n_in columns, 0 after.
struct InputNorm {
    float lo[64], inv_span[64];
};

__global__ void pack_inputs_kernel(const float *theta, int B, int n_in, int ld_out,
                                   __nv_bfloat16 *x, const __grid_constant__ InputNorm nm) {
    const int r = blockIdx.x, c = threadIdx.x;
    if (r >= B || c >= ld_out) return;
    float v = 0.0f;
    if (c < n_in) v = 2.0f * (theta[(size_t)r * n_in + c] - nm.lo[c]) * nm.inv_span[c] - 1.0f;
    x[(size_t)r * ld_out + c] = __float2bfloat16_rn(v);
}

__global__ void hist_to_target_kernel(const uint32_t *h, size_t n, int poisson, float *y) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = poisson ? (float)h[i] : log1pf((float)h[i]);
}

// dZ of the output layer in BF16, its transpose, and the loss sum.  Squared error:
// l = (yhat - y)^2 / 2, dl/dyhat = yhat - y.  Poisson deviance of a log-rate output (targets are
// counts): l = exp(yhat) - y yhat, dl/dyhat = exp(yhat) - y.  Both divided by B.
__global__ void loss_grad_kernel(const float *yhat, const float *y, int B, int N, float inv_b,
                                 int poisson, __nv_bfloat16 *dz, __nv_bfloat16 *dzt, double *loss) {
    __shared__ float tile[kTT][kTT + 1];
    const int n0 = blockIdx.x * kTT, b0 = blockIdx.y * kTT;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    double l = 0.0;
    for (int j = ty; j < kTT; j += 8) {
        const int b = b0 + j, n = n0 + tx;
        float g = 0.0f;
        if (b < B && n < N) {
            const float yh = yhat[(size_t)b * N + n], yt = y[(size_t)b * N + n];
            if (poisson) {
                const float r = expf(yh);
                l += (double)r - (double)yt * (double)yh;
                g = (r - yt) * inv_b;
            } else {
                const float d = yh - yt;
                l += 0.5 * (double)d * (double)d;
                g = d * inv_b;
            }
            dz[(size_t)b * N + n] = __float2bfloat16_rn(g);
        }
        tile[j][tx] = g;
    }
    __syncthreads();
    for (int j = ty; j < kTT; j += 8) {
        const int n = n0 + j, b = b0 + tx;
        if (n < N && b < B) dzt[(size_t)n * B + b] = __float2bfloat16_rn(tile[tx][j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (tx == 0) atomicAdd(loss, l * inv_b);
}

// dZ = dA * gelu'(Z) for a hidden layer, with its transpose.
__global__ void gelu_bwd_kernel(const float *da, const __nv_bfloat16 *z, int B, int N,
                                __nv_bfloat16 *dz, __nv_bfloat16 *dzt) {
    __shared__ float tile[kTT][kTT + 1];
    const int n0 = blockIdx.x * kTT, b0 = blockIdx.y * kTT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int j = ty; j < kTT; j += 8) {
        const int b = b0 + j, n = n0 + tx;
        float g = 0.0f;
        if (b < B && n < N) {
            g = da[(size_t)b * N + n] * gelu_grad(__bfloat162float(z[(size_t)b * N + n]));
            dz[(size_t)b * N + n] = __float2bfloat16_rn(g);
        }
        tile[j][tx] = g;
    }
    __syncthreads();
    for (int j = ty; j < kTT; j += 8) {
        const int n = n0 + j, b = b0 + tx;
        if (n < N && b < B) dzt[(size_t)n * B + b] = __float2bfloat16_rn(tile[tx][j]);
    }
}

// out [C][R] = in [R][C] (BF16, row strides ld_in / ld_out).
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *in, int R, int C, int ld_in,
                                      __nv_bfloat16 *out, int ld_out) {
    __shared__ __nv_bfloat16 tile[kTT][kTT + 2];
    const int c0 = blockIdx.x * kTT, r0 = blockIdx.y * kTT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int j = ty; j < kTT; j += 8) {
        const int r = r0 + j, c = c0 + tx;
        tile[j][tx] = (r < R && c < C) ? in[(size_t)r * ld_in + c] : __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int j = ty; j < kTT; j += 8) {
        const int c = c0 + j, r = r0 + tx;
        if (c < C && r < R) out[(size_t)c * ld_out + r] = tile[tx][j];
    }
}

// db[n] = sum_b dZ^T[n][b]: one warp per row.
__global__ void row_sum_kernel(const __nv_bfloat16 *dzt, int N, int B, float *db) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= N) return;
    float s = 0.0f;
    for (int b = lane; b < B; b += 32) s += __bfloat162float(dzt[(size_t)w * B + b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[w] = s;
}

// Adam on W [N][K] (FP32 master, FP32 moments) with the BF16 copies W [N][K] and W^T [K][N].
__global__ void adam_w_kernel(float *w, float *m, float *v, const float *g, int N, int K, float lr,
                              float b1, float b2, float c1, float c2, float eps,
                              __nv_bfloat16 *wb, __nv_bfloat16 *wt) {
    __shared__ float tile[kTT][kTT + 1];
    const int k0 = blockIdx.x * kTT, n0 = blockIdx.y * kTT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int j = ty; j < kTT; j += 8) {
        const int n = n0 + j, k = k0 + tx;
        float nw = 0.0f;
        if (n < N && k < K) {
            const size_t i = (size_t)n * K + k;
            const float gi = g[i];
            const float mi = b1 * m[i] + (1.0f - b1) * gi;
            const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
            m[i] = mi;
            v[i] = vi;
            nw = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
            w[i] = nw;
            wb[i] = __float2bfloat16_rn(nw);
        }
        tile[j][tx] = nw;
    }
    __syncthreads();
    for (int j = ty; j < kTT; j += 8) {
        const int k = k0 + j, n = n0 + tx;
        if (k < K && n < N) wt[(size_t)k * N + n] = __float2bfloat16_rn(tile[tx][j]);
    }
}

__global__ void adam_b_kernel(float *b, float *m, float *v, const float *g, int N, float lr, float b1,
                              float b2, float c1, float c2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    b[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Surrogate Poisson log-likelihood of each predicted diagram against the data (Section 2.5's
// Poisson alternative): the predicted counts of a model image `scale` times the network's
// image, mh = max(counts * scale, 1/2) * N_d / N_m; sum d ln mh - mh - ln Gamma(d+1).
// The data term sum ln Gamma(d+1) does not depend on the prediction: one block computes it
// once per call (FP64); the per-bin terms are FP32, summed in FP64.
__global__ void data_lgamma_kernel(const uint32_t *data, int N, double *part) {
    __shared__ double ws[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const uint32_t d = data[i];
        if (d > 1u) acc += lgamma((double)d + 1.0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        part[blockIdx.x] = t;
    }
}

// The block partials of data_lgamma_kernel added in a fixed order.
__global__ void sum_partials_kernel(const double *part, int n, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < n; ++k) t += part[k];
        *out = t;
    }
}

__global__ void surrogate_loglike_kernel(const float *yhat, int N, const uint32_t *data, const LLConsts k,
                                         int poisson, const double *lg_sum, double *ll) {
    __shared__ double ws[32];
    const int r = blockIdx.x;
    const float *y = yhat + (size_t)r * N;
    double acc = 0.0;
    if ((N & 3) == 0) {
        const float4 *y4 = reinterpret_cast<const float4 *>(y);
        const uint4 *d4 = reinterpret_cast<const uint4 *>(data);
        for (int i = threadIdx.x; i < (N >> 2); i += blockDim.x) {
            const float4 v = __ldg(y4 + i);
            const uint4 d = __ldg(d4 + i);
            float t = surrogate_ll_term(v.x, d.x, k, poisson);
            t += surrogate_ll_term(v.y, d.y, k, poisson);
            t += surrogate_ll_term(v.z, d.z, k, poisson);
            t += surrogate_ll_term(v.w, d.w, k, poisson);
            acc += (double)t;
        }
    } else {
        for (int i = threadIdx.x; i < N; i += blockDim.x)
            acc += (double)surrogate_ll_term(__ldg(y + i), __ldg(data + i), k, poisson);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        ll[r] = t - *lg_sum;
    }
}

// Fused path: the output layer's epilogue left one partial sum per (row, 64-column block);
// they are added in a fixed order (no atomics, so the result does not depend on scheduling).
__global__ void ll_partials_kernel(const double *part, int ld, int B, const double *lg_sum, double *ll) {
    // one warp per row: coalesced reads, lane-strided sums, then a fixed shuffle tree
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= B) return;
    double t = 0.0;
    for (int k = lane; k < ld; k += 32) t += part[(size_t)r * ld + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) ll[r] = t - *lg_sum;
}

template <class T>
struct Dev {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count) {
        n = count;
        return cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
    }
};

}  // namespace

struct pcmd_mlp {
    int n_layers = 0;
    std::vector<int> dims;       // [n_layers + 1], dims[0] = padded input width
    int n_in = 0;                // raw input features (<= dims[0])
    int max_batch = 0;
    cudaStream_t st = nullptr;
    InputNorm norm;
    struct Layer {
        Dev<float> w, b, mw, vw, mb, vb, gw, gb;
        Dev<__nv_bfloat16> wb, wt;
    };
    std::vector<Layer> L;
    std::vector<Dev<__nv_bfloat16>> x, xt, z;   // x[l]: input of layer l [B][dims[l]]
    Dev<__nv_bfloat16> dz, dzt;
    Dev<float> da, yhat, target, theta;
    Dev<double> loss;
    Dev<uint32_t> err;
    Dev<double> ll;
    Dev<double> ll_part;         // [max_batch][ll_ld] partial likelihood sums (fused path)
    int ll_ld = 0;
    int step = 0;
    int poisson = 0;   // 1: log-rate output trained with the Poisson deviance on counts
    std::string err_text;
};

#define MCK(call)                                                                 \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            mlp->err_text = std::string(#call) + ": " + cudaGetErrorString(e_);   \
            return e_ == cudaErrorMemoryAllocation ? PCMD_ERR_OOM : PCMD_ERR_CUDA; \
        }                                                                         \
    } while (0)

static dim3 tgrid(int cols, int rows) { return dim3((cols + kTT - 1) / kTT, (rows + kTT - 1) / kTT); }

extern "C" {

pcmd_status pcmd_mlp_create(const int *h_dims, int n_layers, int n_in, const float *h_in_lo,
                            const float *h_in_hi, int max_batch, uint64_t seed, void *stream,
                            pcmd_mlp **out) {
    if (!out || !h_dims || n_layers < 1 || n_layers > 16 || max_batch < 1 || max_batch > 65536)
        return PCMD_ERR_ARG;
    *out = nullptr;
    for (int l = 0; l <= n_layers; ++l)
        if (h_dims[l] < 8 || (h_dims[l] & 7) || h_dims[l] > 65536) return PCMD_ERR_ARG;
    if (n_in < 1 || n_in > h_dims[0] || h_dims[0] > 64 || (max_batch & 7)) return PCMD_ERR_ARG;
    pcmd_mlp *mlp = new pcmd_mlp();
    mlp->n_layers = n_layers;
    mlp->dims.assign(h_dims, h_dims + n_layers + 1);
    mlp->n_in = n_in;
    mlp->max_batch = max_batch;
    mlp->st = (cudaStream_t)stream;
    for (int i = 0; i < 64; ++i) {
        mlp->norm.lo[i] = i < n_in && h_in_lo ? h_in_lo[i] : 0.0f;
        const float span = i < n_in && h_in_lo && h_in_hi ? h_in_hi[i] - h_in_lo[i] : 2.0f;
        mlp->norm.inv_span[i] = span != 0.0f ? 1.0f / span : 0.0f;
    }
    // LeCun-normal weights from a seeded Mersenne twister with Box-Muller, zero biases.
    std::mt19937_64 rng(seed);
    auto normal = [&]() {
        const double u1 = ((rng() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((rng() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    mlp->L.resize(n_layers);
    pcmd_status rc = PCMD_OK;
    for (int l = 0; l < n_layers && rc == PCMD_OK; ++l) {
        const int K = mlp->dims[l], N = mlp->dims[l + 1];
        auto &Ly = mlp->L[l];
        const size_t nw = (size_t)N * K;
        std::vector<float> w(nw, 0.0f);
        const int k_real = (l == 0) ? n_in : K;
        const double sd = 1.0 / std::sqrt((double)k_real);
        for (int n = 0; n < N; ++n)
            for (int k = 0; k < k_real; ++k) w[(size_t)n * K + k] = (float)(sd * normal());
        if (Ly.w.alloc(nw) || Ly.b.alloc(N) || Ly.mw.alloc(nw) || Ly.vw.alloc(nw) || Ly.mb.alloc(N) ||
            Ly.vb.alloc(N) || Ly.gw.alloc(nw) || Ly.gb.alloc(N) || Ly.wb.alloc(nw) || Ly.wt.alloc(nw)) {
            rc = PCMD_ERR_OOM;
            break;
        }
        cudaMemcpy(Ly.w.p, w.data(), nw * 4, cudaMemcpyHostToDevice);
        cudaMemset(Ly.b.p, 0, N * 4);
        cudaMemset(Ly.mw.p, 0, nw * 4);
        cudaMemset(Ly.vw.p, 0, nw * 4);
        cudaMemset(Ly.mb.p, 0, N * 4);
        cudaMemset(Ly.vb.p, 0, N * 4);
        // BF16 copies through an Adam step with zero learning rate (writes W and W^T)
        cudaMemset(Ly.gw.p, 0, nw * 4);
        adam_w_kernel<<<tgrid(K, N), dim3(kTT, 8)>>>(Ly.w.p, Ly.mw.p, Ly.vw.p, Ly.gw.p, N, K, 0.0f, 0.9f,
                                                      0.999f, 1.0f, 1.0f, 1e-8f, Ly.wb.p, Ly.wt.p);
    }
    const int B = max_batch;
    mlp->x.resize(n_layers + 1);
    mlp->xt.resize(n_layers);
    mlp->z.resize(n_layers);
    size_t dmax = 0;
    for (int l = 0; l <= n_layers; ++l) dmax = std::max<size_t>(dmax, mlp->dims[l]);
    for (int l = 0; l <= n_layers && rc == PCMD_OK; ++l) {
        if (mlp->x[l].alloc((size_t)B * mlp->dims[l])) rc = PCMD_ERR_OOM;
        if (l < n_layers && (mlp->xt[l].alloc((size_t)B * mlp->dims[l]) || mlp->z[l].alloc((size_t)B * mlp->dims[l + 1])))
            rc = PCMD_ERR_OOM;
    }
    const int dout = mlp->dims[n_layers];
    if (rc == PCMD_OK &&
        (mlp->dz.alloc((size_t)B * dmax) || mlp->dzt.alloc((size_t)B * dmax) || mlp->da.alloc((size_t)B * dmax) ||
         mlp->yhat.alloc((size_t)B * dout) || mlp->target.alloc((size_t)B * dout) ||
         mlp->theta.alloc((size_t)B * 64) || mlp->loss.alloc(1) || mlp->err.alloc(1) || mlp->ll.alloc((size_t)B + 1)))
        rc = PCMD_ERR_OOM;
    mlp->ll_ld = kGemmLlBlocks * ((dout + kGemmTileN - 1) / kGemmTileN);
    if (rc == PCMD_OK && mlp->ll_part.alloc((size_t)B * mlp->ll_ld + 64))
        rc = PCMD_ERR_OOM;
    if (rc == PCMD_OK) {
        cudaMemset(mlp->err.p, 0, 4);
        cudaMemset(mlp->x[0].p, 0, (size_t)B * mlp->dims[0] * 2);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = PCMD_ERR_CUDA;
    }
    if (rc != PCMD_OK) {
        pcmd_mlp_destroy(mlp);
        return rc;
    }
    *out = mlp;
    return PCMD_OK;
}

void pcmd_mlp_destroy(pcmd_mlp *mlp) {
    if (!mlp) return;
    cudaStreamSynchronize(mlp->st);
    for (auto &Ly : mlp->L) {
        Ly.w.release(); Ly.b.release(); Ly.mw.release(); Ly.vw.release(); Ly.mb.release();
        Ly.vb.release(); Ly.gw.release(); Ly.gb.release(); Ly.wb.release(); Ly.wt.release();
    }
    for (auto &d : mlp->x) d.release();
    for (auto &d : mlp->xt) d.release();
    for (auto &d : mlp->z) d.release();
    mlp->dz.release(); mlp->dzt.release(); mlp->da.release(); mlp->yhat.release();
    mlp->target.release(); mlp->theta.release(); mlp->loss.release(); mlp->err.release();
    mlp->ll.release();
    mlp->ll_part.release();
    delete mlp;
}

const char *pcmd_mlp_last_error(const pcmd_mlp *mlp) { return mlp ? mlp->err_text.c_str() : "no network"; }

// Inputs: raw parameters (host or device FP32 [B][n_in]) normalised into x[0].
static pcmd_status stage_inputs(pcmd_mlp *mlp, const float *theta, int B, bool on_device) {
    const float *src = theta;
    if (!on_device) {
        MCK(cudaMemcpyAsync(mlp->theta.p, theta, sizeof(float) * B * mlp->n_in, cudaMemcpyHostToDevice, mlp->st));
        src = mlp->theta.p;
    }
    pack_inputs_kernel<<<B, 64, 0, mlp->st>>>(src, B, mlp->n_in, mlp->dims[0], mlp->x[0].p, mlp->norm);
    MCK(cudaGetLastError());
    return PCMD_OK;
}

static pcmd_status forward(pcmd_mlp *mlp, int B, bool train) {
    for (int l = 0; l < mlp->n_layers; ++l) {
        const int K = mlp->dims[l], N = mlp->dims[l + 1];
        const bool last = l == mlp->n_layers - 1;
        GemmArgs g;
        g.aux = (last || !train) ? nullptr : mlp->z[l].p;   // pre-activations: backward only
        g.bias = mlp->L[l].b.p;
        g.m = B;
        g.n = N;
        g.k = K;
        g.ldc = N;
        g.err = mlp->err.p;
        g.c = last ? (void *)mlp->yhat.p : (void *)mlp->x[l + 1].p;
        MCK(launch_gemm_bf16(mlp->x[l].p, K, mlp->L[l].wb.p, K, g, last ? kEpiBiasF32 : kEpiBiasGeluBf16, mlp->st));
        if (train) {
            transpose_bf16_kernel<<<tgrid(K, B), dim3(kTT, 8), 0, mlp->st>>>(mlp->x[l].p, B, K, K, mlp->xt[l].p, B);
            MCK(cudaGetLastError());
        }
    }
    return PCMD_OK;
}

pcmd_status pcmd_mlp_forward(pcmd_mlp *mlp, const float *theta, int on_device, int B, float *d_out) {
    if (!mlp || !theta || B < 1 || B > mlp->max_batch || (B & 7)) return PCMD_ERR_ARG;
    pcmd_status rc = stage_inputs(mlp, theta, B, on_device != 0);
    if (rc != PCMD_OK) return rc;
    rc = forward(mlp, B, false);
    if (rc != PCMD_OK) return rc;
    if (d_out) {
        MCK(cudaMemcpyAsync(d_out, mlp->yhat.p, sizeof(float) * B * mlp->dims[mlp->n_layers],
                            cudaMemcpyDeviceToDevice, mlp->st));
    }
    return PCMD_OK;
}

pcmd_status pcmd_mlp_targets(pcmd_mlp *mlp, const uint32_t *d_hess, int B) {
    if (!mlp || !d_hess || B < 1 || B > mlp->max_batch) return PCMD_ERR_ARG;
    const size_t n = (size_t)B * mlp->dims[mlp->n_layers];
    hist_to_target_kernel<<<1024, 256, 0, mlp->st>>>(d_hess, n, mlp->poisson, mlp->target.p);
    MCK(cudaGetLastError());
    return PCMD_OK;
}

pcmd_status pcmd_mlp_set_targets(pcmd_mlp *mlp, const float *d_y, int B) {
    if (!mlp || !d_y || B < 1 || B > mlp->max_batch) return PCMD_ERR_ARG;
    MCK(cudaMemcpyAsync(mlp->target.p, d_y, sizeof(float) * B * mlp->dims[mlp->n_layers],
                        cudaMemcpyDeviceToDevice, mlp->st));
    return PCMD_OK;
}

// One optimisation step on the batch whose inputs and targets were staged.
static pcmd_status backward_and_update(pcmd_mlp *mlp, int B, float lr, int update) {
    const int Lc = mlp->n_layers;
    const int dout = mlp->dims[Lc];
    MCK(cudaMemsetAsync(mlp->loss.p, 0, sizeof(double), mlp->st));
    loss_grad_kernel<<<tgrid(dout, B), dim3(kTT, 8), 0, mlp->st>>>(mlp->yhat.p, mlp->target.p, B, dout,
                                                                   1.0f / (float)B, mlp->poisson, mlp->dz.p,
                                                                   mlp->dzt.p, mlp->loss.p);
    MCK(cudaGetLastError());
    for (int l = Lc - 1; l >= 0; --l) {
        const int K = mlp->dims[l], N = mlp->dims[l + 1];
        auto &Ly = mlp->L[l];
        // dW = dZ^T X : A = dZ^T [N][B], B' = X^T [K][B]
        GemmArgs g;
        g.c = Ly.gw.p;
        g.aux = nullptr;
        g.bias = nullptr;
        g.m = N;
        g.n = K;
        g.k = B;
        g.ldc = K;
        g.err = mlp->err.p;
        MCK(launch_gemm_bf16(mlp->dzt.p, B, mlp->xt[l].p, B, g, kEpiF32, mlp->st));
        row_sum_kernel<<<(N * 32 + 255) / 256, 256, 0, mlp->st>>>(mlp->dzt.p, N, B, Ly.gb.p);
        MCK(cudaGetLastError());
        if (l > 0) {
            // dA_{l-1} = dZ W : A = dZ [B][N], B' = W^T [K][N]
            GemmArgs h;
            h.c = mlp->da.p;
            h.aux = nullptr;
            h.bias = nullptr;
            h.m = B;
            h.n = K;
            h.k = N;
            h.ldc = K;
            h.err = mlp->err.p;
            MCK(launch_gemm_bf16(mlp->dz.p, N, Ly.wt.p, N, h, kEpiF32, mlp->st));
            gelu_bwd_kernel<<<tgrid(K, B), dim3(kTT, 8), 0, mlp->st>>>(mlp->da.p, mlp->z[l - 1].p, B, K,
                                                                       mlp->dz.p, mlp->dzt.p);
            MCK(cudaGetLastError());
        }
        if (update) {
            // the update of layer l happens after its dX used the old W^T
            const int t = mlp->step + 1;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.0f / (1.0f - std::pow(b1, (float)t));
            const float c2 = 1.0f / (1.0f - std::pow(b2, (float)t));
            adam_w_kernel<<<tgrid(K, N), dim3(kTT, 8), 0, mlp->st>>>(Ly.w.p, Ly.mw.p, Ly.vw.p, Ly.gw.p, N, K, lr,
                                                                     b1, b2, c1, c2, 1e-8f, Ly.wb.p, Ly.wt.p);
            adam_b_kernel<<<(N + 255) / 256, 256, 0, mlp->st>>>(Ly.b.p, Ly.mb.p, Ly.vb.p, Ly.gb.p, N, lr, b1, b2,
                                                                 c1, c2, 1e-8f);
            MCK(cudaGetLastError());
        }
    }
    if (update) mlp->step++;
    return PCMD_OK;
}

pcmd_status pcmd_mlp_train_step(pcmd_mlp *mlp, const float *theta, int on_device, int B, float lr,
                                int update) {
    if (!mlp || !theta || B < 8 || B > mlp->max_batch || (B & 7)) return PCMD_ERR_ARG;
    pcmd_status rc = stage_inputs(mlp, theta, B, on_device != 0);
    if (rc != PCMD_OK) return rc;
    rc = forward(mlp, B, true);
    if (rc != PCMD_OK) return rc;
    return backward_and_update(mlp, B, lr, update);
}

pcmd_status pcmd_mlp_loss(pcmd_mlp *mlp, double *h_loss) {
    if (!mlp || !h_loss) return PCMD_ERR_ARG;
    MCK(cudaMemcpyAsync(h_loss, mlp->loss.p, sizeof(double), cudaMemcpyDeviceToHost, mlp->st));
    MCK(cudaStreamSynchronize(mlp->st));
    uint32_t e = 0;
    MCK(cudaMemcpy(&e, mlp->err.p, 4, cudaMemcpyDeviceToHost));
    if (e) {
        mlp->err_text = "a bounded wait inside a GEMM ran out";
        return PCMD_ERR_TIMEOUT;
    }
    return PCMD_OK;
}

// sum ln Gamma(d + 1) of the data into ll[max_batch]: block partials in ll_part (rows B..),
// then one fixed-order sum.
static cudaError_t data_lgamma_sum(pcmd_mlp *mlp, const uint32_t *d_data, int N) {
    constexpr int kBlocks = 64;
    double *part = mlp->ll_part.p + (size_t)mlp->max_batch * mlp->ll_ld;
    data_lgamma_kernel<<<kBlocks, 256, 0, mlp->st>>>(d_data, N, part);
    sum_partials_kernel<<<1, 32, 0, mlp->st>>>(part, kBlocks, mlp->ll.p + mlp->max_batch);
    return cudaGetLastError();
}

pcmd_status pcmd_mlp_loglike(pcmd_mlp *mlp, int B, const uint32_t *d_data_hess, double scale, double ratio,
                             double *h_ll) {
    if (!mlp || !d_data_hess || !h_ll || B < 1 || B > mlp->max_batch) return PCMD_ERR_ARG;
    if (!(scale > 0.0) || !(ratio > 0.0)) return PCMD_ERR_ARG;
    const int N = mlp->dims[mlp->n_layers];
    MCK(data_lgamma_sum(mlp, d_data_hess, N));
    surrogate_loglike_kernel<<<B, 256, 0, mlp->st>>>(mlp->yhat.p, N, d_data_hess, ll_consts(scale, ratio), mlp->poisson,
                                                     mlp->ll.p + mlp->max_batch, mlp->ll.p);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(h_ll, mlp->ll.p, sizeof(double) * B, cudaMemcpyDeviceToHost, mlp->st));
    MCK(cudaStreamSynchronize(mlp->st));
    return PCMD_OK;
}

pcmd_status pcmd_mlp_forward_loglike(pcmd_mlp *mlp, const float *theta, int on_device, int B,
                                     const uint32_t *d_data_hess, double scale, double ratio, double *h_ll) {
    if (!mlp || !theta || !d_data_hess || !h_ll || B < 1 || B > mlp->max_batch || (B & 7)) return PCMD_ERR_ARG;
    if (!(scale > 0.0) || !(ratio > 0.0) || ((uintptr_t)d_data_hess & 15)) return PCMD_ERR_ARG;
    pcmd_status rc = stage_inputs(mlp, theta, B, on_device != 0);
    if (rc != PCMD_OK) return rc;
    const int Lc = mlp->n_layers;
    for (int l = 0; l < Lc; ++l) {
        const int K = mlp->dims[l], N = mlp->dims[l + 1];
        GemmArgs g;
        g.bias = mlp->L[l].b.p;
        g.m = B;
        g.n = N;
        g.k = K;
        g.ldc = N;
        g.err = mlp->err.p;
        if (l < Lc - 1) {
            g.c = mlp->x[l + 1].p;
            MCK(launch_gemm_bf16(mlp->x[l].p, K, mlp->L[l].wb.p, K, g, kEpiBiasGeluBf16, mlp->st));
        } else {
            g.ll_data = d_data_hess;
            g.ll_part = mlp->ll_part.p;
            g.ll_ld = mlp->ll_ld;
            g.ll_poisson = mlp->poisson;
            g.llk = ll_consts(scale, ratio);
            MCK(launch_gemm_bf16(mlp->x[l].p, K, mlp->L[l].wb.p, K, g, kEpiPoissonLL, mlp->st));
        }
    }
    const int N = mlp->dims[Lc];
    MCK(data_lgamma_sum(mlp, d_data_hess, N));
    ll_partials_kernel<<<(B + 7) / 8, 256, 0, mlp->st>>>(mlp->ll_part.p, mlp->ll_ld, B,
                                                             mlp->ll.p + mlp->max_batch, mlp->ll.p);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(h_ll, mlp->ll.p, sizeof(double) * B, cudaMemcpyDeviceToHost, mlp->st));
    MCK(cudaStreamSynchronize(mlp->st));
    uint32_t e = 0;
    MCK(cudaMemcpy(&e, mlp->err.p, 4, cudaMemcpyDeviceToHost));
    if (e) {
        mlp->err_text = "a bounded wait inside a GEMM ran out";
        return PCMD_ERR_TIMEOUT;
    }
    return PCMD_OK;
}

// Host copies of layer l's FP32 master weights [N][K] and bias [N] (checkpoints, tests).
pcmd_status pcmd_mlp_get_layer(pcmd_mlp *mlp, int l, float *h_w, float *h_b, float *h_gw, float *h_gb) {
    if (!mlp || l < 0 || l >= mlp->n_layers) return PCMD_ERR_ARG;
    const size_t nw = (size_t)mlp->dims[l] * mlp->dims[l + 1];
    const size_t nb = mlp->dims[l + 1];
    MCK(cudaStreamSynchronize(mlp->st));
    if (h_w) MCK(cudaMemcpy(h_w, mlp->L[l].w.p, nw * 4, cudaMemcpyDeviceToHost));
    if (h_b) MCK(cudaMemcpy(h_b, mlp->L[l].b.p, nb * 4, cudaMemcpyDeviceToHost));
    if (h_gw) MCK(cudaMemcpy(h_gw, mlp->L[l].gw.p, nw * 4, cudaMemcpyDeviceToHost));
    if (h_gb) MCK(cudaMemcpy(h_gb, mlp->L[l].gb.p, nb * 4, cudaMemcpyDeviceToHost));
    return PCMD_OK;
}

pcmd_status pcmd_mlp_set_layer(pcmd_mlp *mlp, int l, const float *h_w, const float *h_b) {
    if (!mlp || l < 0 || l >= mlp->n_layers || !h_w || !h_b) return PCMD_ERR_ARG;
    const int K = mlp->dims[l], N = mlp->dims[l + 1];
    const size_t nw = (size_t)N * K;
    auto &Ly = mlp->L[l];
    MCK(cudaStreamSynchronize(mlp->st));
    MCK(cudaMemcpy(Ly.w.p, h_w, nw * 4, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(Ly.b.p, h_b, (size_t)N * 4, cudaMemcpyHostToDevice));
    MCK(cudaMemset(Ly.gw.p, 0, nw * 4));
    adam_w_kernel<<<tgrid(K, N), dim3(kTT, 8), 0, mlp->st>>>(Ly.w.p, Ly.mw.p, Ly.vw.p, Ly.gw.p, N, K, 0.0f, 1.0f,
                                                             1.0f, 1.0f, 1.0f, 1e-8f, Ly.wb.p, Ly.wt.p);
    MCK(cudaGetLastError());
    return PCMD_OK;
}

pcmd_status pcmd_mlp_set_loss(pcmd_mlp *mlp, int poisson) {
    if (!mlp || (poisson != 0 && poisson != 1)) return PCMD_ERR_ARG;
    mlp->poisson = poisson;
    return PCMD_OK;
}

// Device pointer of the last forward pass's output [B][d_out] FP32.
const float *pcmd_mlp_output(const pcmd_mlp *mlp) { return mlp ? mlp->yhat.p : nullptr; }

pcmd_status pcmd_gemm_bf16(const void *d_a, int lda, const void *d_b, int ldb, void *d_c, int ldc,
                           const float *d_bias, void *d_aux, int m, int n, int k, int epilogue,
                           uint32_t *d_err, void *stream) {
    if (!d_a || !d_b || !d_c || !d_err || m <= 0 || n <= 0 || k <= 0 || ldc < n) return PCMD_ERR_ARG;
    if ((epilogue == PCMD_GEMM_BIAS_F32 || epilogue == PCMD_GEMM_BIAS_GELU_BF16 ||
         epilogue == PCMD_GEMM_BIAS_BF16) && !d_bias)
        return PCMD_ERR_ARG;
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

}  // extern "C"
