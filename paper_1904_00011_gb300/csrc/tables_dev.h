// Device table builder of libpcmd: layout of one model's table and the launch arguments.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "pcmd_internal.h"

namespace pcmd {

// Byte offsets inside one model's table (fixed by P and the band count: every list has room
// for its worst case, so the layout needs no count from the device).
struct TabLayout {
    uint64_t grp_off[2];    // group records of the sparse inversion groups, G per half
    uint64_t dense_off[2];  // group records of the dense inversion groups, G per half
    uint64_t slow_off[2];   // SlowRec[16 G] per half
    uint64_t ptrs_off[2];   // PtrsRec[P] per half
    uint64_t tail_off;      // uint32 [2][16 G][kTailCap] tail thresholds (a fixed slot per point)
    uint64_t flux_off;      // float [P][B] electrons per star
    uint64_t pool_off[2];   // total-count sampler regions (written only when the sampler is used)
    uint64_t bytes;         // table size (256-byte multiple)
};

// Per-model input, computed on the host in FP64.
struct TabSetIn {
    uint64_t base;          // byte offset of the model's table in the table buffer
    double flux_factor;     // 10^(-0.4 dmod)
    uint32_t w_off;         // first weight w_jk = SFH_j MDF_k of the model in `weights`
    int32_t m1_k;           // M1 interpolated isochrone: the grid slot it replaces, or -1
    uint32_t m1_off;        // its first point in `m1_imf` (n_ages * n_mass points per model)
    uint32_t pad;
};

struct TabArgs {
    uint8_t *tables;
    uint8_t *btab;              // word tables of the dense groups, or nullptr (no dense groups)
    uint32_t *err;              // latched error word of the context (kErrBounds)
    SetDesc *desc;              // list lengths are written here (device)
    const TabSetIn *sets;       // [n_sets]
    const double *weights;      // [n_sets][n_ages * n_feh]
    const double *imf;          // [P] IMF weight of each point (per context)
    const double *base_flux;    // [P][B] electrons per star at distance modulus 0 (per context)
    const double *m1_imf;       // [models with M1 interpolation][n_ages][n_mass] IMF weights
    const double *m1_flux;      //   [..][n_ages][n_mass][B] electrons per star at modulus 0
    double hf[2];               // dust-half factors of lambda: (1, 0), (0, 1) or (1 - F, F)
    uint32_t P, G;
    int n_mass, n_feh, n_bands;
    TabLayout layout;
    uint4 *scratch;             // [n_sets][2][G]
    float *insp_lam;            // optional parity copies of model 0: lambda [2][P]
    float *insp_flux;           //   flux [P][B]
    uint32_t *insp_z0;          //   Z_0 [2][P] (0xFFFFFFFF unless 0 < lambda < 640)
    int pool;                   // also build the total-count sampler regions
    uint4 *pool_scratch;        // [n_sets][2][G] pool entries and fixed-point sums (pool only)
    uint4 *pt_scratch;          // [n_sets][2][16 G] per point: Z_0, Z_1, tail length, class
};

TabLayout tab_layout(uint32_t P, int n_bands);
cudaError_t launch_build_tables(const TabArgs &a, int n_sets, cudaStream_t st);

}  // namespace pcmd
