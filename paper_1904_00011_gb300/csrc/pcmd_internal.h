// Internal layouts shared by the host table builder and the kernels of libpcmd.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

namespace pcmd {

constexpr int kMaxBands = 4;
constexpr int kGroup = 16;                // isochrone points per HI call (one byte each)
constexpr float kPtrsThreshold = 640.0f;  // inversion below, transformed rejection at/above
constexpr int kInvCap = 1024;             // inversion counts are capped at 1024 (P(n > 1024) < 2^-140
                                          // for every lambda below 640)
// Threshold slot per inversion point: Z'_0, Z'_1, ... up to the first saturated one (at most 322
// words below a mean of 640: the CDF passes 1 - 2^-33 within 321 counts of the first
// non-negative threshold).
constexpr int kTailCap = 352;
// The total-count sampler draws its per-pixel total by inversion only below 10: a single draw
// per pixel and half would otherwise need one serial FP64 threshold series of up to ~120 terms
// per model and a walk of up to ~60 thresholds per pixel.
constexpr float kPoolTotalLimit = 10.0f;
constexpr float kDenseLam = 0.08f;        // groups with a slot at or above this are "dense"
constexpr uint32_t kPtrsMaxAttempts = 1024u;

// RNG stream kinds (tag = kind << 28 | half << 27 | sub)
enum : uint32_t { kKindHi = 1u, kKindLo = 2u, kKindPtrs = 3u, kKindDust = 4u, kKindNoise = 5u };

// device error bits
enum : uint32_t { kErrSampler = 1u, kErrTimeout = 2u, kErrBounds = 4u };

// Fast-path record of 16 consecutive isochrone points of one dust half (staged in shared memory
// by bulk copies).  Size 64 + 64 * B bytes (a multiple of 16).
//   u32 gid              group index (points 16*gid .. 16*gid+15)
//   u32 pad[3]
//   u32 z7[4]            coarse thresholds zc_j = Z_0 >> 24, slot j at byte j & 3 of word j >> 2,
//                        low 7 bits of each byte
//   u32 zh[4]            the same bytes' top bits (zc_j & 0x80)
//   u8  zc1[16]          Z_1 >> 24 per slot: a certain hit with zc_j < byte < zc1_j has n = 1
//   f32 flux[16][B]      electrons per star of each slot
// Slot j "may be non-zero" iff its HI byte >= zc_j; the 16 tests are four SIMD-within-a-word
// byte compares against z7 / zh.
__host__ __device__ constexpr uint32_t group_rec_bytes(int nb) { return 64u + 64u * (uint32_t)nb; }
constexpr uint32_t kRecZ7 = 16, kRecZh = 32, kRecZc1 = 48, kRecFlux = 64;
// A dense group record holds each slot's leading count n0 (u16[16]) in place of the coarse bytes z7
// and their top bits zh.
constexpr uint32_t kRecN0 = kRecZ7;
// The sparse list (streamed through shared memory) keeps only the first 64 bytes of a record:
// its drain reads a hit's fluxes from the per-point flux table instead.
constexpr uint32_t kSparseRecBytes = 64;

// Slow-path record per point and half (global memory): full 32-bit thresholds.
// The first n0 thresholds of a mean above ~22 are -1 (e^-lambda 2^32 < 1/2: every word exceeds
// them); the record holds the rest, Z'_k = Z_{n0 + k}, and n = n0 + #{k : x > Z'_k}.
struct SlowRec {
    uint32_t z0, z1;        // Z'_0, Z'_1: n > n0 + k  <=>  x > Z'_k
    uint32_t tail_off;      // index of Z'_2 in the tail array
    uint32_t tail_len;      // bits 0-9: number of Z'_k, k >= 2, below 0xFFFFFFFF; bits 10-19: n0;
                            // bits 20-31: start index of the device's threshold walk
};
__host__ __device__ constexpr uint32_t slow_len(uint32_t w) { return w & 0x3FFu; }
__host__ __device__ constexpr uint32_t slow_n0(uint32_t w) { return (w >> 10) & 0x3FFu; }
__host__ __device__ constexpr uint32_t slow_ks(uint32_t w) { return w >> 20; }
__host__ __device__ constexpr uint32_t slow_pack(uint32_t len, uint32_t n0, uint32_t ks) {
    return len | (n0 << 10) | (ks << 20);
}

// Transformed-rejection record (lambda >= 640), 48 bytes.
struct PtrsRec {
    uint32_t i;             // canonical point index
    float lam, b, a, twoa, vr, log_ia;
    float flux[kMaxBands];
    uint32_t pad;
};
static_assert(sizeof(PtrsRec) == 48, "PtrsRec layout");

// Per-set descriptor (device memory).  Offsets are bytes from the start of the table buffer.
struct __align__(16) SetDesc {
    uint64_t grp_off[2];    // group records of half 0 / 1
    uint64_t slow_off[2];   // SlowRec[P] of half 0 / 1
    uint64_t tail_off;      // uint32 tail thresholds
    uint64_t ptrs_off[2];   // PtrsRec lists
    uint64_t img_off;       // float offset of the raw image [B][n][n]
    uint64_t dense_off[2];  // group records of the dense inversion groups (global memory)
    uint32_t n_grp[2], n_ptrs[2], n_dense[2];
    uint32_t n_im, set_id;
    uint32_t item_begin, n_items;   // work items (pixel tiles) of this set
    float dust_a;           // ln(10) * log_ebv
    float dust_sigma;
    float dust_c[kMaxBands];  // -0.4 R_b: factor_b = 10^(dust_c[b] * E)
    uint32_t dust_on;
    uint32_t pool_on;       // total-count sampler for the points below lambda 10
    uint64_t pool_off[2];   // PoolHdr + thresholds / guide / entries per half (host-built)
    uint64_t flux_off;      // float [P][B] electrons per star of every point
    uint64_t btab_off[2];   // word tables of the dense groups (byte offsets in the word-table buffer)
    uint32_t btab_cap;      // dense groups per half the word tables have room for
    uint32_t pad_btab[3];
};

// Word table of a dense group: for each of its 16 slots and each HI byte b one 32-bit entry with a
// count c relative to the slot's n0 (the count at the byte's lower edge, count(b << 24) - n0),
// the threshold Z_(n0 + c) (its bits inside the byte; all ones when the count is the same over
// the whole byte) and a flag set when two or more thresholds fall inside the byte (then c is
// the byte's most frequent count and the thresholds decide from there).  Two layouts, one per
// group (dense record header word 1):
//   narrow (every slot's mean below kWideLam: c - n0 <= 119): bits 0-6 c, bit 7 the flag, bits
//     8-31 the low 24 bits of the threshold; a word x of the byte has count n0 + c + (low24(x) >
//     bits 8-31) unless the flag is set;
//   wide (a mean of kWideLam or more, up to 640: c - n0 <= 222): bits 0-7 c, bits 8-30 bits 1-23
//     of the threshold, bit 31 the flag; equal bits 1-23 (1 word in 2^23) compare x with the
//     threshold itself.
// kBtabGroupBytes per group.
constexpr float kWideLam = 192.0f;
constexpr uint32_t kBtabGroupEntries = kGroup * 256u;
constexpr uint32_t kBtabGroupBytes = kBtabGroupEntries * 4u;

// Total-count sampler of one dust half (the pool = every point with 0 < lambda < 640): header,
// then Z[kInvCap] (inversion thresholds of Lambda, mode 1) or one PtrsRec (mode 2), then the guide
// table (guide[b] = first entry j with T_j > b 2^(32 - bits), guide[2^bits] = n - 1), the pool's
// point indices and their star-assignment thresholds T_j.
constexpr int kPoolGuideBits = 14;
struct __align__(16) PoolHdr {
    float lam;              // (float) Lambda
    uint32_t n;             // pool size
    uint32_t n_z;           // thresholds of the total (mode 1)
    uint32_t mode;          // bits 0-7: 0 empty, 1 inversion (Lambda < 10), 2 transformed
                            // rejection; bits 8-15 (inversion): leading thresholds of -1, n0
};
constexpr uint32_t kPoolZOff = 16, kPoolPtrsOff = kPoolZOff + 4 * kInvCap, kPoolGuideOff = kPoolPtrsOff + 48;
constexpr uint32_t kPoolIdxOff = kPoolGuideOff + 4 * ((1u << kPoolGuideBits) + 4);   // guide[2^bits + 1]
// ... followed by the pool's fixed-point total (uint64, in a 16-byte slot)
constexpr double kPoolFix = 1099511627776.0;   // 2^40: fixed-point scale of the pool weights
__host__ __device__ constexpr uint64_t pool_fix_off(uint32_t P) { return ((kPoolIdxOff + 8ull * P) + 15) & ~15ull; }
__host__ __device__ constexpr uint64_t pool_region_bytes(uint32_t P) { return pool_fix_off(P) + 16; }

// Constants of the pixel stage (noise, magnitudes, Hess binning).
struct PixelConsts {
    float sky[kMaxBands];
    float t[kMaxBands];        // exposure times
    float zp[kMaxBands];       // zero-points, FP32 part
    float zp_lo[kMaxBands];    // zero-points minus their FP32 part
    float c_lo, m_lo, inv_w;   // Hess axes (FP32 bin rule)
    int nx, ny;
    int noise;
    uint64_t seed;
};

struct DrawArgs {
    const uint8_t *tables;      // table buffer
    const uint8_t *btab;        // word tables of the dense groups (full instantiation only)
    const SetDesc *desc;        // [n_sets]
    const uint2 *items;         // (set index, tile) per work item, grouped by set
    const uint32_t *order;      // queue position -> item (longest first); nullptr = identity
    uint32_t n_items;
    uint32_t *queue;            // persistent work counter (nullptr = one item per CTA)
    uint64_t seed;
    uint32_t rk0[10], rk1[10];  // Philox round keys: seed words + r * Weyl constants
    float *image;               // raw images (IMAGE mode)
    uint32_t *counts;           // COUNTS mode output [n_pix][2][P]
    uint32_t count_pix0, count_npix, n_points;
    uint32_t *err;              // device error word
    int chunk;                  // groups per staged chunk (<= 256)
    int split;                  // warps-groups sharing one pixel
    uint32_t ptrs_cap;          // transformed-rejection attempts per draw before the error
    // FUSED mode (no PSF): histogram outputs
    uint32_t *hess;             // [n_sets][ny][nx]
    uint32_t *counters;         // [n_sets][2]
    double *item_moments;       // [n_items][3]
    PixelConsts pc;
};

// PSF / noise / magnitude / Hess stage over raw images.
struct HessArgs {
    const float *image;         // raw images
    const SetDesc *desc;        // for n_im, set_id, img_off; nullptr: one image described by
    uint32_t one_n_im, one_set_id;  //   these two values (image at offset 0)
    int n_sets, n_bands;
    const float *psf;           // device [B][S][S] (or [16][B][S][S] with psf_grid 4), or nullptr
    int psf_in_param;           // nonzero: no device copy, the [B][S][S] weights are the launch's
                                //   host weight array (packed, S = psf_size), passed by value
    int psf_size;
    int psf_grid;               // 1, or 4: a 4x4 grid of regions with their own kernels
    uint32_t *hess;             // [n_sets][ny][nx]
    uint32_t *counters;         // [n_sets][2]
    double *cta_moments;        // [n_sets][ctas_per_set][3]
    int ctas_per_set;
    float *pixels;              // optional [n_sets][B+2][n^2] (packed like the images, B+2 planes)
    const uint64_t *pix_off;    // float offsets of each set's pixel output
    PixelConsts pc;
};

// Draw paths compiled into a draw kernel instantiation besides the sparse inversion groups:
// dense groups + transformed rejection, and the total-count sampler (which replaces the inversion
// groups).  The host launches the smallest set the staged models can need.
enum { kPathSparse = 0, kPathDense = 1, kPathPool = 2 };

// launchers (implemented in the .cu files)
cudaError_t launch_draw(const DrawArgs &a, int n_bands, bool kahan, int mode, int paths, int grid,
                        int block, size_t smem, cudaStream_t st);
int draw_max_blocks_per_sm(int nb, bool kahan, int mode, int paths, int block, size_t smem);
size_t draw_smem_bytes(int n_bands, int chunk, int block, int split, int mode, int nx, int ny);
enum { kModeImage = 0, kModeCounts = 1, kModeFused = 2 };

cudaError_t launch_hess(const HessArgs &a, const float *psf25_host, cudaStream_t st);
size_t hess_smem_bytes(int n_bands, int psf_size, int nx, int ny);
int hess_tiles(int n_im);   // output tiles of an n_im x n_im image in the Hess stage
cudaError_t launch_bin_mags(const float *mag, const float *col, const uint8_t *valid, uint32_t n,
                            uint32_t *hess, uint32_t *counters, double *moments,
                            const PixelConsts &pc, uint32_t *err, cudaStream_t st);
// sums per-CTA / per-item partial moments of each set, in a fixed order, into moments[s][3]
cudaError_t launch_moments_finalize(const double *partials, const uint32_t *part_begin,
                                    const uint32_t *part_count, int n_sets, double *moments,
                                    cudaStream_t st);
// one set whose partials are partials[0 .. count) (range passed by value)
cudaError_t launch_moments_finalize_one(const double *partials, uint32_t count, double *moments,
                                        cudaStream_t st);
// CTAs per set of the likelihood (several when few sets leave SMs idle); `part` holds
// [n_sets][ctas] partial sums, `ticket` [n_sets] counters that are zero between launches.
int loglike_ctas_per_set(int n_sets, int nbins);
cudaError_t launch_loglike(const uint32_t *hess, const double *moments, const SetDesc *desc,
                           int n_sets, int nbins, const uint32_t *mock, double mock_sc,
                           double mock_sm, double mock_nv, double mock_npix, int mode,
                           int sqrtsum, double *part, uint32_t *ticket, double *ll, cudaStream_t st);
cudaError_t upload_stirlerr(const float *tab16);

}  // namespace pcmd
