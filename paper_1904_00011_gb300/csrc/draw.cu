// Launch side of draw_flux (the kernel itself is in draw_kernel.cuh): the sparse-only and
// total-count-sampler instantiations live in this translation unit, those with dense groups and
// transformed rejection in draw_full.cu (the two compile in parallel).
#include "draw_kernel.cuh"

namespace pcmd {

// implemented in draw_full.cu
cudaError_t upload_stirlerr_full(const float *tab16);
int occupancy_full(int paths, int nb, bool kahan, int mode, int block, size_t smem);
cudaError_t launch_full(const DrawArgs &a, int paths, int nb, bool kahan, int mode, int grid, int block,
                        size_t smem, cudaStream_t st);

cudaError_t upload_stirlerr(const float *tab16) {
    const cudaError_t e = upload_stirlerr_local(tab16);
    return e != cudaSuccess ? e : upload_stirlerr_full(tab16);
}

size_t draw_smem_bytes(int nb, int chunk, int block, int split, int mode, int nx, int ny) {
    (void)nb;
    size_t s = 32 + chunk_region_bytes((uint32_t)chunk, kSparseRecBytes) +
               (size_t)kQueueCap * block * 4 +
               (size_t)block * 2 * nb * 4;
    if (mode == kModeFused) {
        s += (size_t)nx * ny * 4 + (size_t)(block / split) * 4;
        s = (s + 7) & ~size_t(7);
        s += (size_t)(block / 32) * 5 * 8 + 8;
    }
    return s;
}

int draw_max_blocks_per_sm(int nb, bool kahan, int mode, int paths, int block, size_t smem) {
    switch (paths) {
        case kPathSparse: return occupancy_paths<kPathSparse>(nb, kahan, mode, block, smem);
        case kPathPool: return occupancy_paths<kPathPool>(nb, kahan, mode, block, smem);
        default: return occupancy_full(paths, nb, kahan, mode, block, smem);
    }
}

cudaError_t launch_draw(const DrawArgs &a, int n_bands, bool kahan, int mode, int paths, int grid, int block,
                        size_t smem, cudaStream_t st) {
    switch (paths) {
        case kPathSparse: return launch_paths<kPathSparse>(a, n_bands, kahan, mode, grid, block, smem, st);
        case kPathPool: return launch_paths<kPathPool>(a, n_bands, kahan, mode, grid, block, smem, st);
        default: return launch_full(a, paths, n_bands, kahan, mode, grid, block, smem, st);
    }
}

}  // namespace pcmd
