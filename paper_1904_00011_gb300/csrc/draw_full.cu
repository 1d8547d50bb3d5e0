// Instantiations of the draw kernel with dense inversion groups and transformed rejection
// (with or without the total-count sampler); see draw_kernel.cuh.
#include "draw_kernel.cuh"

namespace pcmd {

cudaError_t upload_stirlerr_full(const float *tab16) { return upload_stirlerr_local(tab16); }

int occupancy_full(int paths, int nb, bool kahan, int mode, int block, size_t smem) {
    return paths == (kPathDense | kPathPool)
               ? occupancy_paths<kPathDense | kPathPool>(nb, kahan, mode, block, smem)
               : occupancy_paths<kPathDense>(nb, kahan, mode, block, smem);
}

cudaError_t launch_full(const DrawArgs &a, int paths, int nb, bool kahan, int mode, int grid, int block,
                        size_t smem, cudaStream_t st) {
    return paths == (kPathDense | kPathPool)
               ? launch_paths<kPathDense | kPathPool>(a, nb, kahan, mode, grid, block, smem, st)
               : launch_paths<kPathDense>(a, nb, kahan, mode, grid, block, smem, st);
}

}  // namespace pcmd
