// pcmd_hess_noalloc: the PSF / noise / magnitude / Hess stage for callers that cannot allocate
// device memory.  Same kernels as pcmd_hess; their scratch (the image descriptor, the per-CTA
// moment partials and their ranges, a device copy of the PSF) lives in one file-scope device
// array instead of context-owned allocations.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/pcmd.h"
#include "pcmd_internal.h"

namespace pcmd {

constexpr int kNoallocMaxCtas = 1024;

struct NoallocScratch {
    SetDesc desc;
    uint32_t part_begin, part_count, pad[2];
    float psf[kMaxBands * 625];
    double partials[kNoallocMaxCtas * 3];
};

// Shared by every call on a device; holds the last call's contents until the process exits.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

struct PsfParam {
    float w[kMaxBands * 625];
};

// Writes the call's descriptor, partial range and PSF copy into the scratch array (the kernel
// parameters carry the values: no host-to-device copy is needed).
__global__ void noalloc_prepare(NoallocScratch *s, uint32_t n_im, uint32_t set_id, uint32_t n_cta,
                                const __grid_constant__ PsfParam psf) {
    const int t = threadIdx.x;
    if (t == 0) {
        memset(&s->desc, 0, sizeof(SetDesc));
        s->desc.n_im = n_im;
        s->desc.set_id = set_id;
        s->desc.img_off = 0;
        s->part_begin = 0;
        s->part_count = n_cta;
    }
    for (int i = t; i < kMaxBands * 625; i += blockDim.x) s->psf[i] = psf.w[i];
}

// Device address of the scratch array on the current device, looked up once per device.
static NoallocScratch *scratch_on_current_device(cudaError_t *err) {
    static std::mutex mu;
    static NoallocScratch *ptr[128] = {nullptr};
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
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        ptr[dev] = static_cast<NoallocScratch *>(p);
    }
    return ptr[dev];
}

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
    if (!(c.hess_width > 0.0)) return PCMD_ERR_ARG;
    if (c.psf && (c.psf_size < 1 || c.psf_size > 25 || (c.psf_size & 1) == 0)) return PCMD_ERR_ARG;
    for (int b = 0; b < c.n_bands; ++b)
        if (!(c.exptime[b] > 0.0) || c.sky[b] < 0.0) return PCMD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    NoallocScratch *s = scratch_on_current_device(&e);
    if (!s) return PCMD_ERR_CUDA;
    int dev = 0, n_sm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PCMD_ERR_CUDA;
    int ctas = std::min(2 * n_sm, hess_tiles(n_im));
    if (ctas > kNoallocMaxCtas) ctas = kNoallocMaxCtas;
    if (ctas < 1) ctas = 1;

    // The PSF, padded to 25x25 (zero weights add exact zeros), travels as a kernel parameter.
    PsfParam w;
    std::memset(&w, 0, sizeof w);
    if (c.psf) {
        const int S = c.psf_size, o = (25 - S) / 2;
        for (int b = 0; b < c.n_bands; ++b)
            for (int u = 0; u < S; ++u)
                for (int v = 0; v < S; ++v)
                    w.w[b * 625 + (u + o) * 25 + (v + o)] = c.psf[((size_t)b * S + u) * S + v];
    }
    noalloc_prepare<<<1, 256, 0, st>>>(s, (uint32_t)n_im, c.set_id, (uint32_t)ctas, w);
    if (cudaGetLastError() != cudaSuccess) return PCMD_ERR_CUDA;
    const int nbins = c.hess_nx * c.hess_ny;
    if (cudaMemsetAsync(d_hess, 0, sizeof(uint32_t) * nbins, st) != cudaSuccess ||
        cudaMemsetAsync(d_counters, 0, sizeof(uint32_t) * 2, st) != cudaSuccess)
        return PCMD_ERR_CUDA;

    HessArgs h;
    std::memset(&h, 0, sizeof h);
    h.image = d_image;
    h.desc = &s->desc;
    h.n_sets = 1;
    h.n_bands = c.n_bands;
    h.psf = c.psf ? s->psf : nullptr;
    h.psf_size = c.psf ? 25 : 0;
    h.hess = d_hess;
    h.counters = d_counters;
    h.cta_moments = s->partials;
    h.ctas_per_set = ctas;
    h.pixels = nullptr;
    h.pix_off = nullptr;
    PixelConsts &pc = h.pc;
    std::memset(&pc, 0, sizeof pc);
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
    if (launch_hess(h, c.psf ? w.w : nullptr, st) != cudaSuccess) return PCMD_ERR_CUDA;
    if (launch_moments_finalize(s->partials, &s->part_begin, &s->part_count, 1, d_moments, st) !=
        cudaSuccess)
        return PCMD_ERR_CUDA;
    return PCMD_OK;
}
