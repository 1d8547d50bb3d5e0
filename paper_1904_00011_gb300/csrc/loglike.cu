// Log-likelihood of model Hess diagrams against a data Hess diagram (Section 2.5), one CTA per
// set, FP64 block reduction over the bins.
//  PAPER   Eq. 2: sum_i -(d_i/N_d - m_i/N_m)^2 / (2 sigma_i^2) + C,
//          Eq. 3: sigma_i = max(sqrt(d_i^2 + m_i^2), 2)  (sqrtsum: max(sqrt(d_i + m_i), 2)),
//          Eq. 4: C = -(C_d - C_m)^2 / (2 0.05^2) - (M_d - M_m)^2 / (2 0.05^2).
//  POISSON sum_i d_i ln mh_i - mh_i - ln Gamma(d_i + 1), mh_i = max(m_i, 1/2) N_d / N_m.
#include "pcmd_internal.h"
#include <math.h>

namespace pcmd {

// Per-bin terms in FP32 where they are well conditioned (sigma^2 = max(d^2 + m^2, 4) needs no
// square root; the fraction difference is formed in FP64), every accumulation in FP64.
__global__ void __launch_bounds__(1024) loglike_kernel(const uint32_t *hess, const double *moments,
                                                       const SetDesc *desc, int nbins,
                                                       const uint32_t *mock, double mock_sc,
                                                       double mock_sm, double mock_nv,
                                                       double mock_npix, int mode, int sqrtsum,
                                                       double *ll) {
    __shared__ double wsum[32];
    const int s = blockIdx.x;
    const double n_m = (double)desc[s].n_im * (double)desc[s].n_im;
    const double n_d = mock_npix;
    const double inv_nd = 1.0 / n_d, inv_nm = 1.0 / n_m, ratio = n_d / n_m;
    const uint32_t *m = hess + (size_t)s * nbins;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
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
            const float sig2 = fmaxf(sqrtsum ? df + mf : df * df + mf * mf, 4.0f);
            const double g = (double)du * inv_nd - (double)mu * inv_nm;
            acc -= (double)(__fdiv_rn((float)(g * g), 2.0f * sig2));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
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

cudaError_t launch_loglike(const uint32_t *hess, const double *moments, const SetDesc *desc,
                           int n_sets, int nbins, const uint32_t *mock, double mock_sc,
                           double mock_sm, double mock_nv, double mock_npix, int mode,
                           int sqrtsum, double *ll, cudaStream_t st) {
    loglike_kernel<<<n_sets, n_sets >= 152 ? 256 : 1024, 0, st>>>(hess, moments, desc, nbins, mock, mock_sc, mock_sm,
                                           mock_nv, mock_npix, mode, sqrtsum, ll);
    return cudaGetLastError();
}

}  // namespace pcmd
