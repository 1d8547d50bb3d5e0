// pcmd_hess_noalloc: the PSF / noise / magnitude / Hess stage for callers that cannot allocate
// device memory.  Same kernels as pcmd_hess.  The image's size and set id and the PSF weights
// travel by value in the kernel parameters; the only scratch, the per-CTA moment partials, lives
// in one file-scope device array instead of a context-owned allocation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/pcmd.h"
#include "pcmd_internal.h"

namespace pcmd {

constexpr int kNoallocMaxCtas = 1024;

// Shared by every call on a device; holds the last call's partials until the process exits.
// Each call writes the partials of its own CTAs before reading them, so nothing needs clearing.
static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxCtas * 3];

// Device address of the partials array on the current device, looked up once per device.
static double *partials_on_current_device(cudaError_t *err) {
    static std::mutex mu;
    static double *ptr[128] = {nullptr};
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 128) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> g(mu);
    if (!ptr[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (*err != cudaSuccess) return nullptr;
        ptr[dev] = static_cast<double *>(p);
    }
    return ptr[dev];
}

static bool fin(double v) { return std::isfinite(v); }

}  // namespace pcmd

using namespace pcmd;

extern "C" pcmd_status pcmd_hess_noalloc(const pcmd_pixel_config *cfg, const float *d_image, int n_im,
                                         uint32_t *d_hess, double *d_moments, uint32_t *d_counters,
                                         void *stream) {
    if (!cfg || !d_image || !d_hess || !d_moments || !d_counters) return PCMD_ERR_ARG;
    const pcmd_pixel_config &c = *cfg;
    if (c.n_bands < 2 || c.n_bands > PCMD_MAX_BANDS) return PCMD_ERR_ARG;
    if (n_im < 1 || n_im > PCMD_NOALLOC_MAX_IM) return PCMD_ERR_ARG;
    if (c.hess_nx < 1 || c.hess_ny < 1 || (long long)c.hess_nx * c.hess_ny > 40000) return PCMD_ERR_ARG;
    if (!(c.hess_width > 0.0) || !fin(c.hess_width) || !fin(c.hess_c_lo) || !fin(c.hess_m_lo))
        return PCMD_ERR_ARG;
    if (c.psf && (c.psf_size < 1 || c.psf_size > 25 || (c.psf_size & 1) == 0)) return PCMD_ERR_ARG;
    for (int b = 0; b < c.n_bands; ++b)
        if (!(c.exptime[b] > 0.0) || !fin(c.exptime[b]) || !fin(c.zeropoint[b]) || !fin(c.sky[b]) ||
            c.sky[b] < 0.0)
            return PCMD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    double *partials = partials_on_current_device(&e);
    if (!partials) return PCMD_ERR_CUDA;
    int dev = 0, n_sm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PCMD_ERR_CUDA;
    int ctas = std::min(2 * n_sm, hess_tiles(n_im));
    if (ctas > kNoallocMaxCtas) ctas = kNoallocMaxCtas;
    if (ctas < 1) ctas = 1;

    // The PSF, packed [B][S][S], travels in the kernel parameters (S = 25 runs the kernel with
    // compile-time weights, other sizes copy the weights into shared memory).
    static thread_local float w[kMaxBands * 625];
    std::memset(w, 0, sizeof w);
    const int S = c.psf ? c.psf_size : 0;
    for (int b = 0; b < (c.psf ? c.n_bands : 0); ++b)
        for (int i = 0; i < S * S; ++i) {
            const float v = c.psf[(size_t)b * S * S + i];
            if (!std::isfinite(v)) return PCMD_ERR_ARG;
            w[b * S * S + i] = v;
        }
    const int nbins = c.hess_nx * c.hess_ny;
    if (cudaMemsetAsync(d_hess, 0, sizeof(uint32_t) * nbins, st) != cudaSuccess ||
        cudaMemsetAsync(d_counters, 0, sizeof(uint32_t) * 2, st) != cudaSuccess)
        return PCMD_ERR_CUDA;

    HessArgs h;
    std::memset(&h, 0, sizeof h);
    h.image = d_image;
    h.desc = nullptr;
    h.one_n_im = (uint32_t)n_im;
    h.one_set_id = c.set_id;
    h.n_sets = 1;
    h.n_bands = c.n_bands;
    h.psf = nullptr;
    h.psf_in_param = c.psf ? 1 : 0;
    h.psf_size = S;
    h.psf_grid = 1;
    h.hess = d_hess;
    h.counters = d_counters;
    h.cta_moments = partials;
    h.ctas_per_set = ctas;
    h.pixels = nullptr;
    h.pix_off = nullptr;
    PixelConsts &pc = h.pc;
    for (int b = 0; b < kMaxBands; ++b) {
        const bool on = b < c.n_bands;
        pc.sky[b] = on ? (float)c.sky[b] : 0.0f;
        pc.t[b] = on ? (float)c.exptime[b] : 1.0f;
        pc.zp[b] = on ? (float)c.zeropoint[b] : 0.0f;
        pc.zp_lo[b] = on ? (float)(c.zeropoint[b] - (double)pc.zp[b]) : 0.0f;
    }
    pc.c_lo = (float)c.hess_c_lo;
    pc.m_lo = (float)c.hess_m_lo;
    pc.inv_w = (float)(1.0 / c.hess_width);
    pc.nx = c.hess_nx;
    pc.ny = c.hess_ny;
    pc.noise = c.noise ? 1 : 0;
    pc.seed = c.seed;
    if (launch_hess(h, c.psf ? w : nullptr, st) != cudaSuccess) return PCMD_ERR_CUDA;
    if (launch_moments_finalize_one(partials, (uint32_t)ctas, d_moments, st) != cudaSuccess)
        return PCMD_ERR_CUDA;
    return PCMD_OK;
}
