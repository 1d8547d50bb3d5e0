/*
 * pcmd.h -- C ABI of the GB300 pixel colour-magnitude-diagram (pCMD) forward model.
 *
 * The model is the one of Cook, Conroy, van Dokkum & Speagle (2019): for every pixel of an
 * N_im x N_im image, draw a Poisson number of stars at every age-[Fe/H]-mass point of the
 * isochrones with mean lambda = SFH weight x MDF weight x IMF weight normalised to Npix
 * (Section 2.1), sum their fluxes per band with dust and distance applied (Section 2.2), convolve
 * with the PSF, add sky and photon noise, convert to magnitudes (Section 2.1, Fig. 1 panels
 * E-F), bin a Hess diagram and score it against data (Section 2.5, Eq. 2-4).
 *
 * Conventions for every entry point:
 *  - Host pointers are marked h_, device pointers d_.  The library never frees a caller's
 *    pointer.  Configuration arrays are copied at pcmd_create; the caller may free them after.
 *  - Work is enqueued on the stream given in pcmd_config.stream (NULL = legacy default stream)
 *    and is asynchronous unless stated otherwise.
 *  - Every function returns PCMD_OK or an error code; nothing throws across the ABI.  Argument
 *    errors are reported before anything is launched.  Errors raised inside kernels (sampler
 *    attempt cap, bounded waits that ran out) are latched in a device word and reported by the
 *    next synchronising call (pcmd_loglike, pcmd_evaluate, pcmd_sync).  pcmd_last_error gives
 *    a text for the last error of a context.
 *  - A context is not thread-safe; use one per host thread.
 *  - The library owns its scratch (tables, raw images, histograms), sized at pcmd_create from
 *    max_im, max_sets and the isochrone grid, on the device current at pcmd_create.
 */
#ifndef PCMD_H
#define PCMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PCMD_MAX_BANDS 4
#define PCMD_MAX_SFH 32
#define PCMD_MAX_PSF 31

typedef int pcmd_status;
enum {
    PCMD_OK = 0,
    PCMD_ERR_ARG = 1,            /* invalid argument (reported before any launch) */
    PCMD_ERR_CUDA = 2,           /* a CUDA runtime call failed, or a device-built list outgrew
                                  * the room reserved for it (an internal error; the message says
                                  * which) */
    PCMD_ERR_OOM = 3,            /* device or pinned-host allocation failed */
    PCMD_ERR_SAMPLER_LIMIT = 4,  /* transformed rejection hit its attempt cap */
    PCMD_ERR_STATE = 5,          /* call order violated (e.g. pcmd_hess before pcmd_simulate) */
    PCMD_ERR_TIMEOUT = 6         /* a bounded wait inside a kernel ran out */
};

/* flags */
enum {
    PCMD_FLAG_DUST = 1,           /* thin dust screen (Section 2.2 E1-E3) */
    PCMD_FLAG_NOISE = 2,          /* sky + photon noise (Section 2.1) */
    PCMD_FLAG_KAHAN = 4,          /* compensated FP32 flux sums (large Npix) */
    PCMD_FLAG_SIGMA_SQRTSUM = 8,  /* Eq. 3 read as max(sqrt(d + m), 2) instead of as printed */
    PCMD_FLAG_POOL = 16           /* total-count sampler for the points with lambda < 640 (the
                                   * Poisson additivity of the Section 2.1 footnote, used in
                                   * reverse): per pixel and dust half N ~ Poisson(sum of
                                   * their lambdas) stars, each assigned to a point with
                                   * probability lambda_i / sum by inverting the cumulative
                                   * weights; the counts have the same joint law (independent
                                   * Poisson) as per-point draws, from a different RNG stream */
};

/* likelihood modes */
enum { PCMD_LL_PAPER = 0, PCMD_LL_POISSON = 1 };

/* Initial mass function of the IMF weights (Section 2.2): a single power law dN/dm ~ m^-imf_slope
 * (Salpeter: 2.35), or Kroupa (2001): slopes 0.3 below 0.08 Msun, 1.3 to 0.5 Msun, 2.3 above,
 * continuous at the breaks (imf_slope unused). */
enum { PCMD_IMF_POWER = 0, PCMD_IMF_KROUPA = 1 };

/* Hyper-parameters (Table 2) and isochrones; copied at pcmd_create. */
typedef struct {
    int n_bands;                 /* 2..PCMD_MAX_BANDS; band 0 = magnitude axis, colour = m1 - m0 */
    int n_ages, n_feh, n_mass;   /* isochrone grid: n_ages <= PCMD_MAX_SFH */
    const double *log_age;       /* h_[n_ages] log10 age of each SFH bin's isochrone (informational) */
    const double *feh_grid;      /* h_[n_feh] [Fe/H] of the isochrones, strictly ascending (Section 2.2) */
    const double *mass;          /* h_[n_ages][n_feh][n_mass] initial masses, ascending, > 0 */
    const double *abs_mag;       /* h_[n_ages][n_feh][n_mass][n_bands] absolute magnitudes */
    double imf_slope;            /* Salpeter 2.35 (Section 2.2) */
    double exptime[PCMD_MAX_BANDS];   /* seconds (Table 2) */
    double zeropoint[PCMD_MAX_BANDS]; /* magnitude giving 1 e-/s */
    double sky[PCMD_MAX_BANDS];       /* sky electrons per pixel (Table 2, default 0) */
    double r_ext[PCMD_MAX_BANDS];     /* A_band / E(B-V) */
    double f_dust;               /* fraction of stars behind the screen (Section 2.2, default 0.5) */
    double mdf_cut;              /* MDF weights below this are dropped (Section 2.2: 1%) */
    const float *psf;            /* h_[n_bands][psf_size][psf_size], centred; NULL = no PSF */
    int psf_size;                /* odd, <= PCMD_MAX_PSF */
    int hess_nx, hess_ny;        /* Hess bins in colour (x) and magnitude (y) */
    double hess_c_lo, hess_m_lo; /* lower edges of the colour and magnitude axes */
    double hess_width;           /* bin width in magnitudes (Section 2.5: 0.05) */
    int max_im;                  /* largest image edge any call will use */
    int max_sets;                /* largest number of parameter sets per call */
    uint64_t seed;               /* Philox key */
    unsigned flags;              /* PCMD_FLAG_* */
    void *stream;                /* cudaStream_t for all work of this context */
    int imf;                     /* PCMD_IMF_POWER (default) or PCMD_IMF_KROUPA */
    int psf_grid;                /* 0 or 1: one PSF per band; 4: sub-pixel PSFs (Section 2.2): the
                                  * image is a 4x4 grid of regions, output pixel (y, x) in region
                                  * (4y/N, 4x/N) (integer division) uses its own kernel, and psf
                                  * holds [16][n_bands][psf_size][psf_size], region r = 4 ry + rx */
} pcmd_config;

/* Free parameters of one model (Table 1): S5 non-parametric SFH, M2/M3 Gaussian MDF, E1-E3
 * dust screen, D2 distance modulus.  feh_sigma <= 0 selects M1 (Section 2.2, single [Fe/H]):
 * every star has [Fe/H] = feh_mean, on an isochrone interpolated between the grid isochrones
 * k and k + 1 around it (feh_grid[k] <= feh_mean < feh_grid[k + 1], t = (feh_mean -
 * feh_grid[k]) / (feh_grid[k + 1] - feh_grid[k])): each mass point's initial mass and absolute
 * magnitudes are (1 - t) x + t y of the same point of the two grid isochrones; outside the grid
 * the end isochrone is used. */
typedef struct {
    double log_sfh[PCMD_MAX_SFH];  /* log10 stars per pixel formed in each age bin (n_ages used) */
    double feh_mean, feh_sigma;
    double log_ebv, dust_sigma;    /* median log10 E(B-V) and log-normal width (0 = fixed screen) */
    double dmod;                   /* distance modulus */
} pcmd_params;

typedef struct pcmd_ctx pcmd_ctx;

/* Create a context on the current device.  Validates cfg (PCMD_ERR_ARG), copies it, builds the
 * parameter-independent tables (IMF weights of every isochrone, Section 2.2) and allocates the
 * library's scratch.  *out receives the context or NULL on error. */
pcmd_status pcmd_create(const pcmd_config *cfg, pcmd_ctx **out);

/* Release everything the context owns.  NULL is ignored. */
void pcmd_destroy(pcmd_ctx *ctx);

/* Text of the last error of ctx (never NULL; "" when none). */
const char *pcmd_last_error(const pcmd_ctx *ctx);

/* Simulate the raw (pre-PSF) images of n_sets models (Section 2.1 panels A-D): weights,
 * Poisson draws per pixel and isochrone point, per-band flux sums, dust and distance.
 *  h_params  [n_sets] parameters; h_n_im [n_sets] image edges (1..max_im).
 *  first_set_id  set s uses RNG set id first_set_id + s (a re-evaluation of the same model with
 *                another set id is an independent realisation, Appendix A).
 *  d_image   optional (NULL allowed) device float buffer receiving the images, set after set,
 *            each [n_bands][n_im][n_im] row-major; the library also keeps its own copy for
 *            pcmd_hess.
 * Asynchronous. */
pcmd_status pcmd_simulate(pcmd_ctx *ctx, const pcmd_params *h_params, int n_sets,
                          const int *h_n_im, uint32_t first_set_id, float *d_image);

/* PSF convolution (periodic boundary), sky + photon noise, magnitudes and the Hess diagram of
 * the images of the last pcmd_simulate (Section 2.1 panels E-F, Section 2.5).
 *  d_hess     optional [n_sets][hess_ny][hess_nx] uint32 counts (row = magnitude bin)
 *  d_moments  optional [n_sets][3] double: sum of colour, sum of magnitude, valid pixels
 *  d_counters optional [n_sets][2] uint32: valid pixels outside the grid, invalid pixels
 *             (a pixel is invalid when band 0 or 1 has non-positive flux after noise)
 *  d_pixels   optional [n_sets][n_bands + 2][n_im^2] float: noisy fluxes per band, magnitude
 *             and colour of every pixel (NaN where invalid); for inspection and tests.
 * The library keeps its own copy of histograms and moments for pcmd_loglike. Asynchronous. */
pcmd_status pcmd_hess(pcmd_ctx *ctx, uint32_t *d_hess, double *d_moments, uint32_t *d_counters,
                      float *d_pixels);

/* Log-likelihood of every set of the last pcmd_hess against a data Hess diagram (Section 2.5).
 *  d_mock_hess    [hess_ny][hess_nx] uint32 data counts
 *  h_mock_moments [3] sum of colour, sum of magnitude, valid pixels of the data
 *  mock_n_pix     total pixels of the data image (N_d of Eq. 2)
 *  mode           PCMD_LL_PAPER: Eq. 2-4 (flag PCMD_FLAG_SIGMA_SQRTSUM selects the
 *                 max(sqrt(d+m),2) reading of Eq. 3); PCMD_LL_POISSON: sum d ln mh - mh -
 *                 ln Gamma(d+1) with mh = max(m, 1/2) N_d / N_m
 *  h_ll           [n_sets] results (host)
 * Synchronises the stream; returns a latched kernel error if one occurred. */
pcmd_status pcmd_loglike(pcmd_ctx *ctx, const uint32_t *d_mock_hess, const double *h_mock_moments,
                         double mock_n_pix, int mode, double *h_ll);

/* pcmd_simulate + pcmd_hess + pcmd_loglike for n_sets models in one call.  Without a PSF the
 * draw, dust, noise, magnitude and histogram steps run fused in one persistent launch over
 * all sets (uneven image sizes share the grid through a work queue) and the launch sequence
 * is replayed from a CUDA graph.  Arguments as above.  Synchronises the stream. */
pcmd_status pcmd_evaluate(pcmd_ctx *ctx, const pcmd_params *h_params, int n_sets,
                          const int *h_n_im, uint32_t first_set_id, const uint32_t *d_mock_hess,
                          const double *h_mock_moments, double mock_n_pix, int mode,
                          double *h_ll);

/* Synchronise the context's stream and report a latched kernel error, if any. */
pcmd_status pcmd_sync(pcmd_ctx *ctx);

/* --------------------------------------------------------------------------------------- */
/* Inspection entry points used by the parity tests.                                       */
/* --------------------------------------------------------------------------------------- */

/* Launch shape of the draw kernel: block threads (32..256, multiple of 32), split = warp
 * groups that divide the isochrone points of one pixel tile (block / split must be a multiple
 * of 32), chunk = point groups per shared-memory stage (1..256).  Results do not depend on
 * the shape (counts are bit-identical; flux sums may differ by FP32 rounding order).  Used by
 * the autotuner. */
pcmd_status pcmd_set_launch(pcmd_ctx *ctx, int block, int split, int chunk);

/* Debug: lower the transformed-rejection sampler's attempt cap per draw (Section 2.1 Poisson
 * draws at lambda >= 640; the sampler's specification caps a draw at 1024 attempts).  cap
 * 1..1024, 0 restores 1024; anything else returns PCMD_ERR_ARG.  A draw that reaches the cap
 * gives 0 stars and latches PCMD_ERR_SAMPLER_LIMIT, returned by the next synchronising call;
 * this lets a caller exercise that error path (a cap of 1 fails about one draw in seven).
 * Counts with the default cap equal the oracle's; with a lower cap they do not. */
pcmd_status pcmd_set_attempt_cap(pcmd_ctx *ctx, int cap);

/* Kernel timing.  While enabled, the library brackets each of its kernel launches with CUDA
 * events recorded on the context's stream and keeps the pairs per kernel kind;
 * pcmd_kernel_times synchronises, returns the summed milliseconds and launch counts of each
 * kind since the last call (h_ms, h_count: [PCMD_KERNEL_KINDS], host) and clears them.  A graph
 * replay of pcmd_evaluate counts as one PCMD_K_GRAPH launch; PCMD_K_TABLES is the device table
 * builder (its three launches as one). */
enum { PCMD_K_DRAW = 0, PCMD_K_HESS = 1, PCMD_K_FINALIZE = 2, PCMD_K_LOGLIKE = 3,
       PCMD_K_GRAPH = 4, PCMD_K_GEMM = 5, PCMD_K_TABLES = 6, PCMD_KERNEL_KINDS = 8 };
pcmd_status pcmd_profile(pcmd_ctx *ctx, int enable);
pcmd_status pcmd_kernel_times(pcmd_ctx *ctx, double *h_ms, int *h_count);

/* Parametric star-formation histories (Section 2.2 S1-S4) on an age grid: fills h_log_sfh[n_bins]
 * with log10 stars per pixel formed in each bin, summing to Npix, for use as pcmd_params.log_sfh.
 * Bins are [log_age_edges[j], log_age_edges[j+1]) in log10 years (n_bins + 1 increasing edges);
 * star formation starts at the oldest edge T0 (formation time t = T0 - age).
 *   PCMD_SFH_SSP          theta = {log10 Npix, log10 age}: all stars in the bin holding the age
 *   PCMD_SFH_CONSTANT     theta = {log10 Npix}: constant rate, bin mass ~ its width in years
 *   PCMD_SFH_TAU          theta = {log10 Npix, tau [Gyr]}: rate ~ exp(-t / tau)
 *   PCMD_SFH_DELAYED_TAU  theta = {log10 Npix, tau [Gyr]}: rate ~ t exp(-t / tau)
 * Bin masses are the closed-form integrals of the rate over each bin.  Empty bins get -30 (no
 * stars).  Host only; PCMD_ERR_ARG on a bad model, theta, edge list or an all-empty grid. */
enum { PCMD_SFH_SSP = 1, PCMD_SFH_CONSTANT = 2, PCMD_SFH_TAU = 3, PCMD_SFH_DELAYED_TAU = 4 };
pcmd_status pcmd_sfh_bins(int model, const double *theta, int n_theta, int n_bins,
                          const double *log_age_edges, double *h_log_sfh);

/* Number of isochrone points P = n_ages * n_feh * n_mass of the context. */
int pcmd_n_points(const pcmd_ctx *ctx);

/* Host copies of one model's tables, as the device table builder computes them for the draw
 * kernel: h_lam [2][P] FP32 Poisson means of the two dust halves (half 1 = behind the screen),
 * h_flux [P][n_bands] FP32 electrons per star, h_z0 [2][P] the 32-bit draw-word threshold above
 * which a draw is non-zero (0xFFFFFFFF unless 0 < lambda < 640).  Any pointer may be NULL.
 * Builds the model's tables on the context's stream (replacing staged tables of an earlier
 * call) and synchronises. */
pcmd_status pcmd_get_tables(pcmd_ctx *ctx, const pcmd_params *h_params, float *h_lam,
                            float *h_flux, uint32_t *h_z0);

/* Star counts of one model for pixels [pix_begin, pix_begin + n_pix) of an n_im image:
 * d_counts [n_pix][2][P] uint32 (pixel, half, point), written by the production draw kernel
 * compiled with a count output.  Asynchronous. */
pcmd_status pcmd_counts(pcmd_ctx *ctx, const pcmd_params *h_params, int n_im, uint32_t set_id,
                        uint32_t pix_begin, uint32_t n_pix, uint32_t *d_counts);

/* Bin n given FP32 (magnitude, colour) pairs with the Hess kernel's bin rule; d_valid [n]
 * nonzero = valid.  Outputs as in pcmd_hess for one set (d_moments, d_counters may be NULL).
 * Asynchronous. */
pcmd_status pcmd_bin_mags(pcmd_ctx *ctx, const float *d_mag, const float *d_colour,
                          const uint8_t *d_valid, uint32_t n, uint32_t *d_hess,
                          uint32_t *d_counters, double *d_moments);

/* --------------------------------------------------------------------------------------- */
/* Allocation-free Hess stage.                                                              */
/* --------------------------------------------------------------------------------------- */

/* Largest image edge pcmd_hess_noalloc accepts. */
#define PCMD_NOALLOC_MAX_IM 8192

/* Pixel-stage settings for pcmd_hess_noalloc (host struct, read during the call). */
typedef struct {
    int n_bands;                       /* 2..PCMD_MAX_BANDS; band 0 = magnitude axis */
    double exptime[PCMD_MAX_BANDS];    /* seconds */
    double zeropoint[PCMD_MAX_BANDS];  /* magnitude giving 1 e-/s */
    double sky[PCMD_MAX_BANDS];        /* sky electrons per pixel */
    int noise;                         /* nonzero: add sky + photon noise */
    uint64_t seed;                     /* Philox key of the noise draws */
    uint32_t set_id;                   /* RNG set id of the image */
    const float *psf;                  /* HOST [n_bands][psf_size][psf_size] or NULL = no PSF */
    int psf_size;                      /* odd, <= 25 */
    int hess_nx, hess_ny;              /* bins in colour and magnitude (nx * ny <= 40000) */
    double hess_c_lo, hess_m_lo, hess_width;
} pcmd_pixel_config;

/* The paper has no counterpart: this entry point exists for callers that may not allocate GPU
 * memory -- for example code running inside a host application whose memory pool already owns
 * the whole device, or a latency-sensitive loop where cudaMalloc / cudaFree would synchronise the
 * device and stall other streams.  It does what pcmd_hess does for one image (periodic PSF
 * convolution, sky and photon noise, magnitudes, Hess diagram, moments) without a context and
 * without allocating: the image size, set id and PSF weights travel in the kernel parameters, and
 * its only working memory is one fixed 24 KB array (per-CTA moment partials) that the library
 * keeps on every device it runs on until the process exits.
 *  cfg        pixel-stage settings (host)
 *  d_image    [n_bands][n_im][n_im] raw fluxes (device, e.g. from pcmd_simulate)
 *  n_im       image edge, 1..PCMD_NOALLOC_MAX_IM; larger images return PCMD_ERR_ARG
 *  d_hess     [hess_ny][hess_nx] uint32 output (device, cleared by the call)
 *  d_moments  [3] double output: sum of colour, sum of magnitude, valid pixels (device)
 *  d_counters [2] uint32 output: valid pixels outside the grid, invalid pixels (device)
 *  stream     cudaStream_t to run on (NULL = legacy default stream)
 * Results equal pcmd_hess's for the same image, settings and set id.  Asynchronous.
 * The first call on each device looks up the array's device address (make that first call
 * before capturing a stream).  All calls on a device share the array: calls that overlap on the
 * GPU (different streams without ordering between them) race and corrupt each other's moments
 * (never their histograms, counters or memory accesses); order them on one stream or with
 * events.  A non-finite setting or PSF weight returns PCMD_ERR_ARG. */
pcmd_status pcmd_hess_noalloc(const pcmd_pixel_config *cfg, const float *d_image, int n_im,
                              uint32_t *d_hess, double *d_moments, uint32_t *d_counters,
                              void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PCMD_H */
