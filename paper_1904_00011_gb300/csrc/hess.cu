// psf_noise_mag_hess: periodic PSF convolution from a shared-memory tile with halo, sky and
// photon noise, magnitudes and colour, and a Hess diagram privatised in shared memory
// (Section 2.1 panels E-F, Section 2.5).  Persistent over 32-wide x 16-tall output tiles of one
// image per blockIdx.y (a 256x256 image gives 128 tiles); each CTA flushes its histogram once
// and writes one moments partial.
#include "common.cuh"

namespace pcmd {

constexpr int kTileW = 32, kTileH = 16;     // output tile; a warp covers 32 columns x 4 rows
constexpr int kHessThreads = 128;           // 4 warps x 4 rows = kTileH

int hess_tiles(int n_im) { return ((n_im + kTileW - 1) / kTileW) * ((n_im + kTileH - 1) / kTileH); }

struct PsfW {
    float w[kMaxBands][625];   // 25x25 weights per band (compile-time indexed: constant bank)
};

template <int B, int KS>
__device__ __forceinline__ float conv_pixel(const float *tile_b, int hx, int ty, int tx,
                                            const float *w, int ks_rt) {
    float acc = 0.0f;
    if (KS > 0) {
        constexpr int R = KS / 2;
#pragma unroll
        for (int u = 0; u < KS; ++u) {
            const float *row = tile_b + (ty + 2 * R - u) * hx + tx + 2 * R;
#pragma unroll
            for (int v = 0; v < KS; ++v) acc = fmaf(w[u * KS + v], row[-v], acc);
        }
    } else {
        const int R = ks_rt / 2;
        for (int u = 0; u < ks_rt; ++u) {
            const float *row = tile_b + (ty + 2 * R - u) * hx + tx + 2 * R;
            for (int v = 0; v < ks_rt; ++v) acc = fmaf(w[u * ks_rt + v], row[-v], acc);
        }
    }
    return acc;
}

// Four vertically adjacent outputs (rows ty0 .. ty0 + 3, column tx) of a KS x KS kernel with
// compile-time weights: every input value read from shared memory feeds up to four outputs.
// The input rows are walked from the bottom up, so each output accumulates its terms in the
// same order as conv_pixel (kernel row u ascending, then column v ascending).
template <int KS>
__device__ __forceinline__ void conv_col4(const float *tile_b, int hx, int ty0, int tx,
                                          const float *w, float out[4]) {
    constexpr int R = KS / 2;
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = 0.0f;
#pragma unroll
    for (int r = KS + 2; r >= 0; --r) {
        const float *row = tile_b + (ty0 + r) * hx + tx + 2 * R;
#pragma unroll
        for (int v = 0; v < KS; ++v) {
            const float x = row[-v];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int u = k + 2 * R - r;
                if (u >= 0 && u < KS) out[k] = fmaf(w[u * KS + v], x, out[k]);
            }
        }
    }
}

// KS: 0 = no PSF, 25 = 25x25 weights from the kernel parameter, -1 = any odd size from smem
// (a single 25x25 PSF runs hess_bs_kernel below).
// GRID: the sub-pixel PSF grid (Section 2.2): output pixel (y, x) takes the kernel of region
// (4y/N, 4x/N), read from global memory (the region is uniform over most warps, so the loads
// are broadcasts from L1).
template <int B, int KS, bool GRID>
__global__ void __launch_bounds__(kHessThreads) hess_kernel(const __grid_constant__ HessArgs a,
                                                            const __grid_constant__ PsfW pw) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int set = blockIdx.y;
    const SetDesc *dp = a.desc ? a.desc + set : nullptr;
    const int N = dp ? (int)dp->n_im : (int)a.one_n_im;
    const uint32_t set_id = dp ? dp->set_id : a.one_set_id;
    const uint64_t img_off = dp ? dp->img_off : 0ull;
    const uint32_t npix = (uint32_t)N * (uint32_t)N;
    const int ks = KS > 0 ? KS : (KS == 0 ? 0 : a.psf_size);
    const int R = ks / 2;
    const int hx = kTileW + 2 * R, hy = kTileH + 2 * R;
    const int nbins = a.pc.nx * a.pc.ny;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
    float *tile = reinterpret_cast<float *>(hist + nbins);
    float *wsm = tile + (KS != 0 ? B * hx * hy : 0);
    double *wred = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(wsm + (KS < 0 ? B * ks * ks : 0)) + 7u) & ~uintptr_t(7));
    const int tid = threadIdx.x;
    for (int i = tid; i < nbins; i += kHessThreads) hist[i] = 0u;
    if (KS < 0 && !GRID)
        for (int i = tid; i < B * ks * ks; i += kHessThreads)
            wsm[i] = a.psf ? a.psf[i] : (&pw.w[0][0])[i];
    __syncthreads();

    const float *img = a.image + img_off;
    float *pout = a.pixels ? a.pixels + a.pix_off[set] : nullptr;
    const int tiles_x = (N + kTileW - 1) / kTileW;
    const int n_tiles = tiles_x * ((N + kTileH - 1) / kTileH);
    double cs = 0.0, ms = 0.0, nv = 0.0;
    uint32_t novf = 0u, ninv = 0u;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int y0 = (t / tiles_x) * kTileH, x0 = (t % tiles_x) * kTileW;
        if (KS != 0) {
            // one warp per halo row, lanes along it; periodic wrap by whole images
            for (int ty = tid >> 5; ty < hy; ty += kHessThreads / 32) {
                int gy = y0 - R + ty;
                while (gy < 0) gy += N;
                while (gy >= N) gy -= N;
                for (int tx = tid & 31; tx < hx; tx += 32) {
                    int gx = x0 - R + tx;
                    while (gx < 0) gx += N;
                    while (gx >= N) gx -= N;
                    const size_t src = (size_t)gy * N + gx;
#pragma unroll
                    for (int b = 0; b < B; ++b) tile[b * hx * hy + ty * hx + tx] = __ldg(img + (size_t)b * npix + src);
                }
            }
            __syncthreads();
        }
        const int tx = tid & 31;
        for (int ty = tid >> 5; ty < kTileH; ty += kHessThreads / 32) {
            const int y = y0 + ty, x = x0 + tx;
            const bool in = y < N && x < N;
            int bin = -1;
            if (in) {
                const uint32_t p = (uint32_t)y * (uint32_t)N + (uint32_t)x;
                float F[B];
                const float *gk = nullptr;
                if (GRID) {
                    const int region = ((4 * y) / N) * 4 + (4 * x) / N;
                    gk = a.psf + (size_t)region * B * ks * ks;
                }
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    if (KS == 0) F[b] = __ldg(img + (size_t)b * npix + p);
                    else if (GRID) F[b] = conv_pixel<B, KS>(tile + b * hx * hy, hx, ty, tx, gk + b * ks * ks, ks);
                    else if (KS > 0) F[b] = conv_pixel<B, KS>(tile + b * hx * hy, hx, ty, tx, pw.w[b], ks);
                    else F[b] = conv_pixel<B, KS>(tile + b * hx * hy, hx, ty, tx, wsm + b * ks * ks, ks);
                }
                const PixelOut o = pixel_stage<B>(F, p, set_id, a.pc);
                if (o.valid) {
                    cs += (double)__fsub_rn(o.col, a.pc.c_lo);
                    ms += (double)__fsub_rn(o.mag, a.pc.m_lo);
                    nv += 1.0;
                    bin = o.bin;
                    if (bin < 0) ++novf;
                } else {
                    ++ninv;
                }
                if (pout) {
#pragma unroll
                    for (int b = 0; b < B; ++b) pout[(size_t)b * npix + p] = F[b];
                    pout[(size_t)B * npix + p] = o.valid ? o.mag : __int_as_float(0x7fc00000);
                    pout[(size_t)(B + 1) * npix + p] = o.valid ? o.col : __int_as_float(0x7fc00000);
                }
            }
            hist_add_warp(hist, nullptr, nullptr, bin, 0u);
        }
        if (KS != 0) __syncthreads();
    }
    __syncthreads();
    uint32_t *gh = a.hess + (size_t)set * nbins;
    for (int i = tid; i < nbins; i += kHessThreads) {
        const uint32_t v = hist[i];
        if (v) atomicAdd(gh + i, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cs += __shfl_xor_sync(0xffffffffu, cs, o);
        ms += __shfl_xor_sync(0xffffffffu, ms, o);
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
        novf += __shfl_xor_sync(0xffffffffu, novf, o);
        ninv += __shfl_xor_sync(0xffffffffu, ninv, o);
    }
    const int wid = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        wred[wid * 3 + 0] = cs;
        wred[wid * 3 + 1] = ms;
        wred[wid * 3 + 2] = nv;
        if (novf) atomicAdd(a.counters + (size_t)set * 2 + 0, novf);
        if (ninv) atomicAdd(a.counters + (size_t)set * 2 + 1, ninv);
    }
    __syncthreads();
    if (tid == 0) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < kHessThreads / 32; ++w) {
            t0 += wred[w * 3 + 0];
            t1 += wred[w * 3 + 1];
            t2 += wred[w * 3 + 2];
        }
        double *out = a.cta_moments + ((size_t)set * a.ctas_per_set + blockIdx.x) * 3;
        out[0] = t0 + t2 * (double)a.pc.c_lo;
        out[1] = t1 + t2 * (double)a.pc.m_lo;
        out[2] = t2;
    }
}

// 4-byte global -> shared copy through the async copy unit (no register staging: every copy of
// a halo tile is in flight at once).
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__host__ __device__ constexpr int bs_halo_w() { return kTileW + 24; }
__host__ __device__ constexpr int bs_halo_h() { return kTileH + 24; }

// The 25x25 PSF stage with the tile's convolutions split over bands: 4 warps per band (4 rows
// each), so a CTA runs 4 B warps.  The halo tile is fetched with one async copy per element from
// wrapped row / column index tables (periodic boundary), the convolved tile meets in shared
// memory, and every thread then runs the pixel stage of 512 / (128 B) pixels.
template <int B>
__global__ void __launch_bounds__(128 * B) hess_bs_kernel(const __grid_constant__ HessArgs a,
                                                          const __grid_constant__ PsfW pw) {
    constexpr int KS = 25, R = KS / 2, HX = bs_halo_w(), HY = bs_halo_h(), NT = 128 * B;
    constexpr int TP = kTileW * kTileH;
    extern __shared__ __align__(16) uint8_t smem[];
    const int set = blockIdx.y;
    const SetDesc *dp = a.desc ? a.desc + set : nullptr;
    const int N = dp ? (int)dp->n_im : (int)a.one_n_im;
    const uint32_t set_id = dp ? dp->set_id : a.one_set_id;
    const uint64_t img_off = dp ? dp->img_off : 0ull;
    const uint32_t npix = (uint32_t)N * (uint32_t)N;
    const int nbins = a.pc.nx * a.pc.ny;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
    float *tile = reinterpret_cast<float *>(hist + nbins);          // [B][HY][HX]
    float *conv = tile + B * HY * HX;                                // [B][kTileH][kTileW]
    int *rowtab = reinterpret_cast<int *>(conv + B * TP);            // [HY] wrapped rows * N
    int *coltab = rowtab + HY;                                       // [HX] wrapped columns
    double *wred = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(coltab + HX) + 7u) & ~uintptr_t(7));
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < nbins; i += NT) hist[i] = 0u;

    const float *img = a.image + img_off;
    float *pout = a.pixels ? a.pixels + a.pix_off[set] : nullptr;
    const int tiles_x = (N + kTileW - 1) / kTileW;
    const int n_tiles = tiles_x * ((N + kTileH - 1) / kTileH);
    double cs = 0.0, ms = 0.0, nv = 0.0;
    uint32_t novf = 0u, ninv = 0u;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int y0 = (t / tiles_x) * kTileH, x0 = (t % tiles_x) * kTileW;
        for (int i = tid; i < HY + HX; i += NT) {
            const int v = (i < HY ? y0 + i : x0 + (i - HY)) - R;
            const int wv = ((v % N) + N) % N;
            if (i < HY) rowtab[i] = wv * N;
            else coltab[i - HY] = wv;
        }
        __syncthreads();
        for (int i = tid; i < B * HY * HX; i += NT) {
            const int b = i / (HY * HX), r = i - b * (HY * HX);
            const int ty = r / HX, tx = r - ty * HX;
            cp_async4(tile + i, img + (size_t)b * npix + (size_t)(rowtab[ty] + coltab[tx]));
        }
        cp_async_wait_all();
        __syncthreads();
        {
            const int b = wid >> 2, ty0 = (wid & 3) * 4;
            float o[4];
#pragma unroll
            for (int bb = 0; bb < B; ++bb)
                if (bb == b) conv_col4<KS>(tile + bb * HY * HX, HX, ty0, lane, pw.w[bb], o);
#pragma unroll
            for (int k = 0; k < 4; ++k) conv[b * TP + (ty0 + k) * kTileW + lane] = o[k];
        }
        __syncthreads();
        for (int q = tid; q < TP; q += NT) {
            const int y = y0 + q / kTileW, x = x0 + (q % kTileW);
            int bin = -1;
            if (y < N && x < N) {
                const uint32_t p = (uint32_t)y * (uint32_t)N + (uint32_t)x;
                float F[B];
#pragma unroll
                for (int b = 0; b < B; ++b) F[b] = conv[b * TP + q];
                const PixelOut o = pixel_stage<B>(F, p, set_id, a.pc);
                if (o.valid) {
                    cs += (double)__fsub_rn(o.col, a.pc.c_lo);
                    ms += (double)__fsub_rn(o.mag, a.pc.m_lo);
                    nv += 1.0;
                    bin = o.bin;
                    if (bin < 0) ++novf;
                } else {
                    ++ninv;
                }
                if (pout) {
#pragma unroll
                    for (int b = 0; b < B; ++b) pout[(size_t)b * npix + p] = F[b];
                    pout[(size_t)B * npix + p] = o.valid ? o.mag : __int_as_float(0x7fc00000);
                    pout[(size_t)(B + 1) * npix + p] = o.valid ? o.col : __int_as_float(0x7fc00000);
                }
            }
            hist_add_warp(hist, nullptr, nullptr, bin, 0u);
        }
        __syncthreads();
    }
    uint32_t *gh = a.hess + (size_t)set * nbins;
    for (int i = tid; i < nbins; i += NT) {
        const uint32_t v = hist[i];
        if (v) atomicAdd(gh + i, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cs += __shfl_xor_sync(0xffffffffu, cs, o);
        ms += __shfl_xor_sync(0xffffffffu, ms, o);
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
        novf += __shfl_xor_sync(0xffffffffu, novf, o);
        ninv += __shfl_xor_sync(0xffffffffu, ninv, o);
    }
    if (lane == 0) {
        wred[wid * 3 + 0] = cs;
        wred[wid * 3 + 1] = ms;
        wred[wid * 3 + 2] = nv;
        if (novf) atomicAdd(a.counters + (size_t)set * 2 + 0, novf);
        if (ninv) atomicAdd(a.counters + (size_t)set * 2 + 1, ninv);
    }
    __syncthreads();
    if (tid == 0) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < NT / 32; ++w) {
            t0 += wred[w * 3 + 0];
            t1 += wred[w * 3 + 1];
            t2 += wred[w * 3 + 2];
        }
        double *out = a.cta_moments + ((size_t)set * a.ctas_per_set + blockIdx.x) * 3;
        out[0] = t0 + t2 * (double)a.pc.c_lo;
        out[1] = t1 + t2 * (double)a.pc.m_lo;
        out[2] = t2;
    }
}

static size_t hess_bs_smem_bytes(int nb, int nx, int ny) {
    size_t s = (size_t)nx * ny * 4 + (size_t)nb * bs_halo_h() * bs_halo_w() * 4 +
               (size_t)nb * kTileW * kTileH * 4 + (size_t)(bs_halo_h() + bs_halo_w()) * 4;
    s = (s + 7) & ~size_t(7);
    s += (size_t)(128 * nb / 32) * 3 * 8;
    return s;
}

template <int B>
static cudaError_t launch_hess_bs(const HessArgs &a, const PsfW &w, cudaStream_t st) {
    static size_t configured = 0;
    const size_t smem = hess_bs_smem_bytes(B, a.pc.nx, a.pc.ny);
    auto k = hess_bs_kernel<B>;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    dim3 grid(a.ctas_per_set, a.n_sets);
    k<<<grid, 128 * B, smem, st>>>(a, w);
    return cudaGetLastError();
}

size_t hess_smem_bytes(int nb, int psf_size, int nx, int ny) {
    const int R = psf_size / 2;
    size_t s = (size_t)nx * ny * 4;
    if (psf_size > 0) s += (size_t)nb * (kTileW + 2 * R) * (kTileH + 2 * R) * 4;
    if (psf_size > 0 && psf_size != 25) s += (size_t)nb * psf_size * psf_size * 4;
    s = (s + 7) & ~size_t(7);
    s += (kHessThreads / 32) * 3 * 8;
    return s;
}

template <int B, int KS, bool GRID>
static cudaError_t launch_hess_t(const HessArgs &a, const PsfW &w, size_t smem, cudaStream_t st) {
    static size_t configured = 0;
    auto k = hess_kernel<B, KS, GRID>;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    dim3 grid(a.ctas_per_set, a.n_sets);
    k<<<grid, kHessThreads, smem, st>>>(a, w);
    return cudaGetLastError();
}

template <int B>
static cudaError_t launch_hess_b(const HessArgs &a, const PsfW &w, size_t smem, cudaStream_t st) {
    if ((!a.psf && !a.psf_in_param) || a.psf_size == 0) return launch_hess_t<B, 0, false>(a, w, smem, st);
    if (a.psf_grid == 4) {
        if (a.psf_size == 25) return launch_hess_t<B, 25, true>(a, w, smem, st);
        return launch_hess_t<B, -1, true>(a, w, smem, st);
    }
    if (a.psf_size == 25) return launch_hess_bs<B>(a, w, st);
    return launch_hess_t<B, -1, false>(a, w, smem, st);
}

// The 25x25 weights travel as a kernel parameter (constant bank, compile-time offsets);
// psf25_host is the context's host copy [kMaxBands][625] (or nullptr).  With psf_in_param the
// same array holds packed [B][S][S] weights of any size S (identical layout for S = 25).
cudaError_t launch_hess(const HessArgs &a, const float *psf25_host, cudaStream_t st) {
    const bool has_psf = (a.psf || a.psf_in_param) && a.psf_size > 0;
    const size_t smem = hess_smem_bytes(a.n_bands, has_psf ? a.psf_size : 0, a.pc.nx, a.pc.ny);
    PsfW w;
    for (int b = 0; b < kMaxBands; ++b)
        for (int i = 0; i < 625; ++i) w.w[b][i] = psf25_host ? psf25_host[b * 625 + i] : 0.0f;
    switch (a.n_bands) {
        case 2: return launch_hess_b<2>(a, w, smem, st);
        case 3: return launch_hess_b<3>(a, w, smem, st);
        default: return launch_hess_b<4>(a, w, smem, st);
    }
}

// ---------------------------------------------------------------------------------------
// Binning of given FP32 (magnitude, colour) pairs with the same rule (parity tests).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) bin_mags_kernel(const float *mag, const float *col,
                                                       const uint8_t *valid, uint32_t n,
                                                       uint32_t *hess, uint32_t *counters,
                                                       double *moments, PixelConsts pc) {
    extern __shared__ uint32_t shist[];
    const int nbins = pc.nx * pc.ny;
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) shist[i] = 0u;
    __syncthreads();
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        int bin = -1;
        if (i < n) {
            if (valid[i]) {
                bin = hess_bin(mag[i], col[i], pc);
                if (moments) {
                    atomicAdd(moments + 0, (double)col[i]);
                    atomicAdd(moments + 1, (double)mag[i]);
                    atomicAdd(moments + 2, 1.0);
                }
                if (bin < 0 && counters) atomicAdd(counters + 0, 1u);
            } else if (counters) {
                atomicAdd(counters + 1, 1u);
            }
        }
        hist_add_warp(shist, nullptr, nullptr, bin, 0u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += blockDim.x)
        if (shist[i]) atomicAdd(hess + i, shist[i]);
}

cudaError_t launch_bin_mags(const float *mag, const float *col, const uint8_t *valid, uint32_t n,
                            uint32_t *hess, uint32_t *counters, double *moments,
                            const PixelConsts &pc, uint32_t *err, cudaStream_t st) {
    (void)err;
    const size_t smem = (size_t)pc.nx * pc.ny * 4;
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(bin_mags_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    int grid = (int)((n + 255) / 256);
    if (grid > 1024) grid = 1024;
    if (grid < 1) grid = 1;
    bin_mags_kernel<<<grid, 256, smem, st>>>(mag, col, valid, n, hess, counters, moments, pc);
    return cudaGetLastError();
}

// One warp per set: lane l adds partials l, l + 32, ... in order, then a fixed xor tree.
// begin == nullptr: one set, partials [0, one_count).
__global__ void moments_finalize_kernel(const double *partials, const uint32_t *begin,
                                        const uint32_t *count, int n_sets, double *moments,
                                        uint32_t one_count) {
    const int s = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    if (s >= n_sets) return;
    const uint32_t lane = threadIdx.x & 31u;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const double *p = partials + (begin ? (size_t)begin[s] * 3 : 0);
    const uint32_t cnt = begin ? count[s] : one_count;
    for (uint32_t i = lane; i < cnt; i += 32u) {
        a0 += p[i * 3 + 0];
        a1 += p[i * 3 + 1];
        a2 += p[i * 3 + 2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
        moments[s * 3 + 0] = a0;
        moments[s * 3 + 1] = a1;
        moments[s * 3 + 2] = a2;
    }
}

cudaError_t launch_moments_finalize(const double *partials, const uint32_t *part_begin,
                                    const uint32_t *part_count, int n_sets, double *moments,
                                    cudaStream_t st) {
    moments_finalize_kernel<<<(n_sets + 3) / 4, 128, 0, st>>>(partials, part_begin, part_count,
                                                             n_sets, moments, 0u);
    return cudaGetLastError();
}

cudaError_t launch_moments_finalize_one(const double *partials, uint32_t count, double *moments,
                                        cudaStream_t st) {
    moments_finalize_kernel<<<1, 32, 0, st>>>(partials, nullptr, nullptr, 1, moments, count);
    return cudaGetLastError();
}

}  // namespace pcmd
