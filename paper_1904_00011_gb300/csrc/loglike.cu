// Log-likelihood of model Hess diagrams against a data Hess diagram (Section 2.5).
//  PAPER   Eq. 2: sum_i -(d_i/N_d - m_i/N_m)^2 / (2 sigma_i^2) + C,
//          Eq. 3: sigma_i = max(sqrt(d_i^2 + m_i^2), 2)  (sqrtsum: max(sqrt(d_i + m_i), 2)),
//          Eq. 4: C = -(C_d - C_m)^2 / (2 0.05^2) - (M_d - M_m)^2 / (2 0.05^2).
//  POISSON sum_i d_i ln mh_i - mh_i - ln Gamma(d_i + 1), mh_i = max(m_i, 1/2) N_d / N_m.
// The bins of a set are split over `ctas` CTAs (more than one when few sets would leave SMs
// idle: FP64 is slow on this GPU, so the work is spread); every CTA reduces its bins in a fixed
// order and writes a partial, and the last CTA of the set to finish (an atomic ticket) adds
// the partials in CTA order and Eq. 4.  The result does not depend on which CTA finishes last.
#include "pcmd_internal.h"
#include <math.h>
#include <algorithm>

namespace pcmd {

constexpr int kLlThreads = 256;

// Sum over the block in a fixed order (warp trees, then the warp sums in order); valid in
// thread 0.
__device__ __forceinline__ double block_sum(double v, double *ws) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    return t;
}

// Per-bin terms: paper mode in FP32 (sigma^2 = max(d^2 + m^2, 4) needs no square root; the
// fraction difference, its square and the quotient are single FP32 operations, accurate to a
// few 1e-7 of each term), Poisson mode in FP64; every accumulation in FP64.
__global__ void __launch_bounds__(kLlThreads) loglike_kernel(const uint32_t *hess, const double *moments,
                                                             const SetDesc *desc, int nbins,
                                                             const uint32_t *mock, double mock_sc,
                                                             double mock_sm, double mock_nv,
                                                             double mock_npix, int mode, int sqrtsum,
                                                             double *part, uint32_t *ticket, double *ll) {
    __shared__ double wsum[kLlThreads / 32];
    __shared__ bool s_last;
    const int s = blockIdx.y, c = blockIdx.x, ctas = gridDim.x;
    const double n_m = (double)desc[s].n_im * (double)desc[s].n_im;
    const double n_d = mock_npix;
    const double ratio = n_d / n_m;
    const float inv_nd = (float)(1.0 / n_d), inv_nm = (float)(1.0 / n_m);
    const uint32_t *m = hess + (size_t)s * nbins;
    const int per = (nbins + ctas - 1) / ctas;
    const int lo = c * per, hi = min(nbins, lo + per);
    double acc = 0.0;
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
        const uint32_t du = __ldg(mock + i), mu = __ldg(m + i);
        if (mode == 1) {
            const double mh = fmax((double)mu, 0.5) * ratio;
            acc -= mh;
            if (du) {
                const double di = (double)du;
                acc += di * log(mh) - lgamma(di + 1.0);
            }
        } else {
            if ((du | mu) == 0u) continue;
            const float df = (float)du, mf = (float)mu;
            const float sig2 = fmaxf(sqrtsum ? __fadd_rn(df, mf) : __fadd_rn(__fmul_rn(df, df), __fmul_rn(mf, mf)), 4.0f);
            const float g = __fsub_rn(__fmul_rn(df, inv_nd), __fmul_rn(mf, inv_nm));
            acc -= (double)__fdiv_rn(__fmul_rn(g, g), __fmul_rn(2.0f, sig2));
        }
    }
    double t = block_sum(acc, wsum);
    if (ctas > 1) {
        if (threadIdx.x == 0) {
            part[(size_t)s * ctas + c] = t;
            __threadfence();
            s_last = atomicAdd(ticket + s, 1u) == (uint32_t)(ctas - 1);
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        double v = 0.0;
        for (int k = (int)threadIdx.x; k < ctas; k += blockDim.x) v += __ldcg(part + (size_t)s * ctas + k);
        __syncthreads();
        t = block_sum(v, wsum);
        if (threadIdx.x == 0) ticket[s] = 0u;            // ready for the next launch
    }
    if (threadIdx.x == 0) {
        if (mode != 1) {
            const double *mo = moments + (size_t)s * 3;
            if (mo[2] <= 0.0 || mock_nv <= 0.0) {
                t = -INFINITY;
            } else {
                const double cd = mock_sc / mock_nv, md = mock_sm / mock_nv;
                const double cm = mo[0] / mo[2], mm = mo[1] / mo[2];
                t += -((cd - cm) * (cd - cm)) / (2.0 * 0.05 * 0.05) -
                     ((md - mm) * (md - mm)) / (2.0 * 0.05 * 0.05);
            }
        }
        ll[s] = t;
    }
}

int loglike_ctas_per_set(int n_sets, int nbins) {
    if (n_sets >= 152) return 1;
    const int by_bins = (nbins + kLlThreads - 1) / kLlThreads;
    const int by_sms = (2 * 152 + n_sets - 1) / n_sets;
    return std::max(1, std::min(by_bins, by_sms));
}

cudaError_t launch_loglike(const uint32_t *hess, const double *moments, const SetDesc *desc,
                           int n_sets, int nbins, const uint32_t *mock, double mock_sc,
                           double mock_sm, double mock_nv, double mock_npix, int mode,
                           int sqrtsum, double *part, uint32_t *ticket, double *ll, cudaStream_t st) {
    const int ctas = loglike_ctas_per_set(n_sets, nbins);
    loglike_kernel<<<dim3(ctas, n_sets), kLlThreads, 0, st>>>(hess, moments, desc, nbins, mock, mock_sc,
                                                              mock_sm, mock_nv, mock_npix, mode, sqrtsum,
                                                              part, ticket, ll);
    return cudaGetLastError();
}

}  // namespace pcmd
