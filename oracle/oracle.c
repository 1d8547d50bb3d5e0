/*
 * pCMD forward-model ORACLE -- test infrastructure only.
 *
 * A plain, slow CPU restatement of the pixel colour-magnitude-diagram forward model of
 * Cook, Conroy, van Dokkum & Speagle (2019), Section 2.1 and Section 2.2, written to check the
 * CUDA path against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load it; the product library never links, calls or reads anything here, and this file
 * includes no header of the product.
 *
 * Precision: weights, fluxes, dust, PSF, noise and magnitudes are FP64.  The Poisson sampler's
 * decisions follow the sampler specification exactly (FP64 CDF for inversion, FP32 IEEE basic
 * operations for transformed rejection) so that star counts can be compared bit for bit.
 * Build with -ffp-contract=off and without -ffast-math: every float operation below is one
 * IEEE-754 round-to-nearest operation in the order written.
 *
 * Sampler specification (the same one the CUDA path implements independently):
 *   RNG      Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011, "Parallel random numbers: as easy
 *            as 1, 2, 3"), key = 64-bit seed, counter = (pixel, index, set, tag).
 *   tag      kind << 28 | half << 27 | sub;  kinds HI=1, LO=2, PTRS=3, DUST=4, NOISE=5.
 *   uniform  u(w) = ((w >> 8) | 1) * 2^-24, exact in FP32, in (0, 1).
 *   inversion (lambda < 640): x = b << 24 | l >> 8 with b byte (i & 3) of word (i & 15) >> 2
 *            of the HI call with index i >> 4, l word (i & 3) of the LO call with index
 *            i >> 2; v = (x + 0.5) 2^-32;
 *            n = min{k : v < F_k}, F_k the FP64 Poisson CDF by p_k = p_{k-1} lambda / k,
 *            capped at 1024.
 *   PTRS (lambda >= 640): Hormann (1993) transformed rejection with squeeze, attempts a use
 *            words 2(a&1), 2(a&1)+1 of the PTRS call with sub = a >> 1; acceptance in the
 *            deviance form of the log-pmf (Loader 2000), all in FP32 with the series log below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------- */
/* Philox4x32-10: round function and key schedule as published by Salmon et al. (2011).   */
/* ------------------------------------------------------------------------------------- */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += OR_PHILOX_W0; k1 += OR_PHILOX_W1; }
        uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    memcpy(out, c, sizeof c);
}

enum { OR_KIND_HI = 1, OR_KIND_LO = 2, OR_KIND_PTRS = 3, OR_KIND_DUST = 4, OR_KIND_NOISE = 5 };

static uint32_t or_tag(uint32_t kind, uint32_t half, uint32_t sub)
{
    return (kind << 28) | (half << 27) | sub;
}

static void or_call(uint64_t seed, uint32_t pix, uint32_t index, uint32_t set, uint32_t tag,
                    uint32_t out[4])
{
    uint32_t ctr[4] = {pix, index, set, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox(ctr, key, out);
}

/* The 32-bit draw word of inversion entry (half, point i) at pixel pix: the top byte from the
 * HI call of the point's group of 16, the low 24 bits from the LO call of its group of 4. */
uint32_t or_draw_word(uint64_t seed, uint32_t pix, uint32_t i, uint32_t set, uint32_t half)
{
    uint32_t whi[4], wlo[4];
    or_call(seed, pix, i >> 4, set, or_tag(OR_KIND_HI, half, 0), whi);
    or_call(seed, pix, i >> 2, set, or_tag(OR_KIND_LO, half, 0), wlo);
    const uint32_t b = (whi[(i & 15u) >> 2] >> (8u * (i & 3u))) & 0xFFu;
    return (b << 24) | (wlo[i & 3u] >> 8);
}

float or_uniform(uint32_t w)
{
    return (float)((w >> 8) | 1u) * 0x1p-24f;
}

/* ------------------------------------------------------------------------------------- */
/* FP32 natural log from basic operations: exponent split, mantissa reduced to            */
/* [sqrt(1/2), sqrt(2)], atanh series ln m = 2 (s + s^3/3 + ... + s^11/11), s=(m-1)/(m+1) */
/* (Abramowitz & Stegun 4.1.27).  Valid for finite normal x > 0.                          */
/* ------------------------------------------------------------------------------------- */
static float or_f32_from_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t or_bits_from_f32(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

float or_lnf(float x)
{
    const float SQRT2 = or_f32_from_bits(0x3FB504F3u);        /* fl32(sqrt 2) */
    const float LN2_HI = 0.693145751953125f;                   /* 45426 / 2^16 */
    const float LN2_LO = (float)(0.69314718055994530942 - 0.693145751953125);
    const float C3 = (float)(1.0 / 3.0), C5 = (float)(1.0 / 5.0), C7 = (float)(1.0 / 7.0);
    const float C9 = (float)(1.0 / 9.0), C11 = (float)(1.0 / 11.0);
    uint32_t u = or_bits_from_f32(x);
    int e = (int)(u >> 23) - 127;
    float m = or_f32_from_bits((u & 0x007FFFFFu) | 0x3F800000u);
    if (m > SQRT2) { m = m * 0.5f; e = e + 1; }
    float num = m - 1.0f;
    float den = m + 1.0f;
    float s = num / den;
    float z = s * s;
    float p = C11;
    p = p * z; p = p + C9;
    p = p * z; p = p + C7;
    p = p * z; p = p + C5;
    p = p * z; p = p + C3;
    float t = s * z;
    t = t * p;
    float lnm = s + t;
    lnm = lnm + lnm;
    float ef = (float)e;
    float hi = ef * LN2_HI;
    float lo = ef * LN2_LO;
    float r = lnm + lo;
    r = r + hi;
    return r;
}

/* ------------------------------------------------------------------------------------- */
/* Poisson sampler                                                                        */
/* ------------------------------------------------------------------------------------- */

/* The sampler's boundary: inversion below, transformed rejection at and above; inversion counts
 * are capped at OR_INV_CAP (P(n > 1024) < 2^-140 for every mean below 640: the CDF passes
 * 1 - 2^-33 first, so the cap never truncates the law). */
#define OR_INV_LIMIT 640.0f
#define OR_INV_CAP 1024u

/* Inversion for lambda < 640: n = min{k : v < F_k}, v = (x + 0.5) 2^-32, FP64 CDF. */
uint32_t or_poisson_inversion(float lam_f, uint32_t x)
{
    double lam = (double)lam_f;
    double p = exp(-lam);
    double F = p;
    double v = ldexp((double)x + 0.5, -32);
    uint32_t k = 0;
    while (v >= F && k < OR_INV_CAP) {
        k = k + 1u;
        p = p * lam;
        p = p / (double)k;
        F = F + p;
    }
    return k;
}

/* Per-point constants of transformed rejection (Hormann 1993), FP64 rounded to FP32. */
typedef struct { float lam, b, a, twoa, vr, log_ia; } or_ptrs_consts;

void or_ptrs_setup(float lam_f, float out6[6])
{
    double lam = (double)lam_f;
    double slam = sqrt(lam);
    double b = 0.931 + 2.53 * slam;
    double a = -0.059 + 0.02483 * b;
    double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
    double vr = 0.9277 - 3.6224 / (b - 2.0);
    out6[0] = lam_f;
    out6[1] = (float)b;
    out6[2] = (float)a;
    out6[3] = (float)(2.0 * a);
    out6[4] = (float)vr;
    out6[5] = (float)log(inv_alpha);
}

/* stirlerr(k) = ln k! - (k ln k - k + 0.5 ln(2 pi k)): FP64 table for k < 16 (from lgamma),
 * FP32 Stirling series 1/(12k) - 1/(360k^3) + 1/(1260k^5) above (DLMF 5.11.1). */
static float or_stirlerr(float kf)
{
    if (kf < 16.0f) {
        double k = (double)kf;
        double s = lgamma(k + 1.0);
        s = s - (k + 0.5) * log(k);
        s = s + k;
        s = s - 0.5 * log(2.0 * M_PI);
        return (float)s;
    }
    const float S1 = (float)(1.0 / 12.0), S2 = (float)(1.0 / 360.0), S3 = (float)(1.0 / 1260.0);
    float r = 1.0f / kf;
    float r2 = r * r;
    float t = r2 * S3;
    t = S2 - t;
    t = t * r2;
    t = S1 - t;
    return t * r;
}

/* phi(x) = (1 + x) ln(1 + x) - x, series sum_{n=2}^{13} (-1)^n x^n / (n (n-1)) for |x| < 1/4. */
static float or_phi(float x)
{
    if (fabsf(x) < 0.25f) {
        float c[14];
        for (int n = 2; n <= 13; ++n)
            c[n] = (float)(((n % 2 == 0) ? 1.0 : -1.0) / ((double)n * ((double)n - 1.0)));
        float p = c[13];
        for (int n = 12; n >= 2; --n) { p = p * x; p = p + c[n]; }
        float r = p * x;
        return r * x;
    }
    float y = 1.0f + x;
    float r = y * or_lnf(y);
    return r - x;
}

/* log Poisson pmf in the deviance form: -lambda phi((k-lambda)/lambda) - 0.5 ln(2 pi k)
 * - stirlerr(k), the form that avoids cancelling k ln lambda against ln k! (Loader 2000). */
float or_log_pmf(float kf, float lam)
{
    if (kf == 0.0f) return -lam;
    const float HALF_LN_2PI = (float)0.91893853320467274178;
    float d = kf - lam;
    float x = d / lam;
    float bd0 = lam * or_phi(x);
    float st = or_stirlerr(kf);
    float t = or_lnf(kf);
    t = 0.5f * t;
    t = t + HALF_LN_2PI;
    float r = -bd0;
    r = r - t;
    r = r - st;
    return r;
}

/* The log-form acceptance test of an attempt the squeeze leaves open (Hormann 1993):
 * ln V + ln inv_alpha - ln q <= log pmf(k), q = a / us^2 + b.  For k >= 1 the pmf's term
 * -ln(k) / 2 moves to the left-hand side, which takes one logarithm: ln(V sqrt(k) / q) +
 * ln inv_alpha <= -lambda phi((k - lambda) / lambda) - ln(2 pi) / 2 - stirlerr(k); k = 0 keeps
 * ln V + ln inv_alpha - ln q <= -lambda.  FP32 basic operations in this order. */
static int or_ptrs_log_accept(float V, float q, float kf, float lam, float log_ia)
{
    if (kf == 0.0f) {
        float lhs = or_lnf(V);
        lhs = lhs + log_ia;
        lhs = lhs - or_lnf(q);
        return lhs <= -lam;
    }
    const float HALF_LN_2PI = (float)0.91893853320467274178;
    float y = V * sqrtf(kf);
    y = y / q;
    float lhs = or_lnf(y);
    lhs = lhs + log_ia;
    float d = kf - lam;
    float x = d / lam;
    float rhs = -(lam * or_phi(x));
    rhs = rhs - HALF_LN_2PI;
    rhs = rhs - or_stirlerr(kf);
    return lhs <= rhs;
}

#define OR_PTRS_MAX_ATTEMPTS 1024u

/* Transformed rejection with squeeze (Hormann 1993) for lambda >= 640.  Returns the count,
 * or UINT32_MAX if the attempt cap is reached. */
uint32_t or_poisson_ptrs(const float c6[6], uint64_t seed, uint32_t pix, uint32_t i,
                         uint32_t set, uint32_t half, uint32_t *attempts_out)
{
    const float lam = c6[0], b = c6[1], a = c6[2], twoa = c6[3], vr = c6[4], log_ia = c6[5];
    uint32_t w[4];
    for (uint32_t at = 0; at < OR_PTRS_MAX_ATTEMPTS; ++at) {
        if ((at & 1u) == 0u) or_call(seed, pix, i, set, or_tag(OR_KIND_PTRS, half, at >> 1), w);
        uint32_t wu = w[2u * (at & 1u)], wv = w[2u * (at & 1u) + 1u];
        float U = or_uniform(wu) - 0.5f;
        float V = or_uniform(wv);
        float us = 0.5f - fabsf(U);
        float t = twoa / us;
        t = t + b;
        t = t * U;
        t = t + lam;
        t = t + 0.43f;
        float kf = floorf(t);
        if (us >= 0.07f && V <= vr) { if (attempts_out) *attempts_out = at + 1; return (uint32_t)kf; }
        if (kf < 0.0f || (us < 0.013f && V > us)) continue;
        if (kf > 1.0e9f) continue;
        float q = us * us;
        q = a / q;
        q = q + b;
        if (or_ptrs_log_accept(V, q, kf, lam, log_ia)) { if (attempts_out) *attempts_out = at + 1; return (uint32_t)kf; }
    }
    if (attempts_out) *attempts_out = OR_PTRS_MAX_ATTEMPTS;
    return UINT32_MAX;
}

/* One Poisson draw of entry (half, i) with FP32 mean lam at pixel pix (Section 2.1: the number
 * of stars of every age-[Fe/H]-mass bin in every pixel is Poisson). */
uint32_t or_draw(float lam, uint64_t seed, uint32_t pix, uint32_t i, uint32_t set, uint32_t half,
                 int *err)
{
    if (lam == 0.0f) return 0u;
    if (lam < OR_INV_LIMIT) return or_poisson_inversion(lam, or_draw_word(seed, pix, i, set, half));
    float c6[6];
    or_ptrs_setup(lam, c6);
    uint32_t n = or_poisson_ptrs(c6, seed, pix, i, set, half, NULL);
    if (n == UINT32_MAX) { if (err) *err = 1; return 0u; }
    return n;
}

/* ------------------------------------------------------------------------------------- */
/* Model weights (Section 2.1, Section 2.2)                                               */
/* ------------------------------------------------------------------------------------- */

/* lambda[j][k][i] = SFH_j * MDF_k * IMF_jk,i in FP64, summing to Npix = sum_j SFH_j.
 *  SFH_j  = 10^log_sfh[j]                      (S5: log stars per pixel formed in bin j)
 *  MDF_k  = Gaussian density at the grid [Fe/H], normalised, weights < mdf_cut removed,
 *           renormalised (M2/M3); feh_sigma <= 0 puts all weight on the nearest grid point
 *           (M1: the Python layer first puts the interpolated isochrone in that slot)
 *  IMF_i  = integral of m^-slope over the mass cell of point i (cells bounded by geometric
 *           midpoints), normalised over the isochrone (Salpeter slope 2.35).  */
/* Kroupa (2001) IMF over [a, b]: dN/dm proportional to m^-0.3 below 0.08 Msun, m^-1.3 from 0.08 to
 * 0.5 Msun and m^-2.3 above, the three pieces joined continuously (factors 1, 0.08, 0.04). */
static double or_kroupa(double a, double b)
{
    const double edge[4] = {0.0, 0.08, 0.5, 1.0e300};
    const double alpha[3] = {0.3, 1.3, 2.3};
    const double join[3] = {1.0, 0.08, 0.04};
    double total = 0.0;
    for (int s = 0; s < 3; ++s) {
        double x0 = a > edge[s] ? a : edge[s];
        double x1 = b < edge[s + 1] ? b : edge[s + 1];
        if (x1 <= x0) continue;
        double p = 1.0 - alpha[s];
        double v = pow(x1, p) - pow(x0, p);
        v = v / p;
        total = total + join[s] * v;
    }
    return total;
}

void or_weights(int n_ages, int n_feh, int n_mass, const double *mass, double slope, int kroupa,
                const double *feh_grid, const double *log_sfh, double feh_mean,
                double feh_sigma, double mdf_cut, double *lam_out)
{
    double *mdf = (double *)calloc((size_t)n_feh, sizeof(double));
    if (feh_sigma > 0.0) {
        double s = 0.0;
        for (int k = 0; k < n_feh; ++k) {
            double t = feh_grid[k] - feh_mean;
            t = t / feh_sigma;
            mdf[k] = exp(-0.5 * (t * t));
            s = s + mdf[k];
        }
        double s2 = 0.0;
        for (int k = 0; k < n_feh; ++k) {
            mdf[k] = mdf[k] / s;
            if (mdf[k] < mdf_cut) mdf[k] = 0.0;
            s2 = s2 + mdf[k];
        }
        for (int k = 0; k < n_feh; ++k) mdf[k] = mdf[k] / s2;
    } else {
        int best = 0;
        for (int k = 1; k < n_feh; ++k)
            if (fabs(feh_grid[k] - feh_mean) < fabs(feh_grid[best] - feh_mean)) best = k;
        mdf[best] = 1.0;
    }
    double *omega = (double *)malloc(sizeof(double) * (size_t)n_mass);
    double *edge = (double *)malloc(sizeof(double) * (size_t)(n_mass + 1));
    for (int j = 0; j < n_ages; ++j) {
        double sfh = pow(10.0, log_sfh[j]);
        for (int k = 0; k < n_feh; ++k) {
            const double *m = mass + ((size_t)j * n_feh + k) * n_mass;
            double s = 0.0;
            if (n_mass == 1) {
                omega[0] = 1.0;
                s = 1.0;
            } else {
                for (int i = 1; i < n_mass; ++i) edge[i] = sqrt(m[i - 1] * m[i]);
                edge[0] = m[0] * m[0] / edge[1];
                edge[n_mass] = m[n_mass - 1] * m[n_mass - 1] / edge[n_mass - 1];
                double a1 = 1.0 - slope;
                for (int i = 0; i < n_mass; ++i) {
                    double w;
                    if (kroupa) {
                        w = or_kroupa(edge[i], edge[i + 1]);
                    } else if (a1 != 0.0) {
                        w = pow(edge[i + 1], a1) - pow(edge[i], a1);
                        w = w / a1;
                    } else {
                        w = log(edge[i + 1] / edge[i]);
                    }
                    omega[i] = w;
                    s = s + w;
                }
            }
            double wjk = sfh * mdf[k];
            double *out = lam_out + ((size_t)j * n_feh + k) * n_mass;
            for (int i = 0; i < n_mass; ++i) out[i] = wjk * (omega[i] / s);
        }
    }
    free(omega);
    free(edge);
    free(mdf);
}

/* Per-star flux in electrons: t_b 10^(-0.4 ((M_b + dmod) - ZP_b)), FP64 (Section 2.1, D1/D2). */
void or_fluxes(int n_pts, int n_bands, const double *abs_mag, double dmod, const double *zp,
               const double *exptime, double *flux_out)
{
    for (int i = 0; i < n_pts; ++i)
        for (int b = 0; b < n_bands; ++b) {
            double s = abs_mag[(size_t)i * n_bands + b] + dmod;
            s = s - zp[b];
            s = -0.4 * s;
            double f = pow(10.0, s);
            flux_out[(size_t)i * n_bands + b] = exptime[b] * f;
        }
}

/* Split lambda between stars in front of (half 0) and behind (half 1) a thin dust screen
 * that reddens a fraction f_dust of the stars (Section 2.2): independent Poisson draws with
 * means (1 - f) lambda and f lambda.  Without dust, or f = 0, only half 0 is drawn; f = 1
 * draws half 1 only.  lam_h[h * n + i] receives FP32 means (0 where a half is unused). */
int or_halves(int n, const double *lam, int dust, double f_dust, float *lam_h)
{
    for (int i = 0; i < n; ++i) {
        double l0, l1;
        if (!dust || f_dust <= 0.0) { l0 = lam[i]; l1 = 0.0; }
        else if (f_dust >= 1.0) { l0 = 0.0; l1 = lam[i]; }
        else { l0 = lam[i] * (1.0 - f_dust); l1 = lam[i] * f_dust; }
        lam_h[i] = (float)l0;
        lam_h[(size_t)n + i] = (float)l1;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Simulation of the raw (pre-PSF) image                                                  */
/* ------------------------------------------------------------------------------------- */

/* Dust screen factors of one pixel (Section 2.2 E1-E3): E(B-V) = 10^log_ebv exp(sigma z),
 * z ~ N(0,1) by Box-Muller from the pixel's DUST call; factor_b = 10^(-0.4 R_b E). */
static void or_dust_factors(uint64_t seed, uint32_t pix, uint32_t set, int n_bands,
                            double log_ebv, double dust_sigma, const double *r_ext, double *fac)
{
    double z = 0.0;
    if (dust_sigma != 0.0) {
        uint32_t w[4];
        or_call(seed, pix, 0, set, or_tag(OR_KIND_DUST, 0, 0), w);
        double u1 = (double)or_uniform(w[0]), u2 = (double)or_uniform(w[1]);
        z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    }
    double ebv = exp(log(10.0) * log_ebv + dust_sigma * z);
    for (int b = 0; b < n_bands; ++b) fac[b] = pow(10.0, -0.4 * r_ext[b] * ebv);
}

/* Raw image [n_bands][n_im][n_im] (FP64) for pixels [pix_begin, pix_end) of one model:
 * per pixel, draws for every entry of both halves, flux sums per band in FP64, the dust factor
 * on the behind half.  counts (optional) receives n for every (pixel, half, point) as
 * counts[(p - pix_begin) * 2 * n_pts + h * n_pts + i].  Returns nonzero on a sampler overrun. */
/* Total-count sampler.  The Section 2.1 footnote states that a sum of Poisson counts is Poisson
 * with the summed mean; the sampler uses the converse (the standard splitting property, not
 * stated in the paper): a Poisson total split over the points by their weights gives
 * independent Poisson counts.  Weights in fixed point: L_i = floor(lambda_i 2^40) for 0 < lambda_i < 640
 * (lambda_i 2^40 is exact in FP64), and the pool of one half is every point with L_i > 0, in
 * point order (the others below 640 draw no star).  C_j = L_0 + ... + L_j and Lfix = C_(n-1)
 * are exact integers; the total's mean is Lambda = (float)(Lfix 2^-40), the FP64 conversion
 * rounding to nearest.  Star assignment thresholds T_j = min(floor(C_j 2^32 / Lfix), 2^32 - 1)
 * in exact integer arithmetic; a star with word u goes to the first pool entry with u < T_j,
 * or to the last. */
typedef struct {
    uint32_t n;            /* pool size */
    uint32_t *idx;         /* point of each pool entry */
    uint32_t *thr;         /* T_j (the last entry's is unused) */
    float lam;             /* Lambda */
} or_pool;

static void or_pool_build(const float *lam, int n_pts, or_pool *pl)
{
    pl->n = 0;
    pl->idx = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n_pts > 0 ? n_pts : 1));
    pl->thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n_pts > 0 ? n_pts : 1));
    uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_pts > 0 ? n_pts : 1));
    uint64_t c = 0;
    for (int i = 0; i < n_pts; ++i) {
        if (!(lam[i] > 0.0f && lam[i] < OR_INV_LIMIT)) continue;
        uint64_t w = (uint64_t)((double)lam[i] * 1099511627776.0);
        if (w == 0) continue;
        c += w;
        pl->idx[pl->n] = (uint32_t)i;
        cum[pl->n] = c;
        pl->n++;
    }
    for (uint32_t j = 0; j < pl->n; ++j) {
        unsigned __int128 q = ((unsigned __int128)cum[j] << 32) / c;
        pl->thr[j] = q >= 0xFFFFFFFFu ? 0xFFFFFFFFu : (uint32_t)q;
    }
    pl->lam = (float)ldexp((double)c, -40);
    free(cum);
}

/* The pool of one half as arrays: n (returned), idx[n], thr[n], *lam_total = Lambda. */
int or_pool_tables(const float *lam, int n_pts, uint32_t *idx, uint32_t *thr, float *lam_total)
{
    or_pool pl;
    or_pool_build(lam, n_pts, &pl);
    for (uint32_t j = 0; j < pl.n; ++j) { idx[j] = pl.idx[j]; thr[j] = pl.thr[j]; }
    *lam_total = pl.lam;
    free(pl.idx);
    free(pl.thr);
    return (int)pl.n;
}

static uint32_t or_pool_pick(const or_pool *pl, uint32_t u)
{
    /* the first j < n - 1 with u < T_j, else n - 1; T_j is non-decreasing, so a bisection over
     * j in [0, n - 1) finds the same entry as the scan in point order */
    uint32_t lo = 0, hi = pl->n - 1u;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2u;
        if (u < pl->thr[mid]) hi = mid;
        else lo = mid + 1u;
    }
    return pl->idx[lo];
}

/* Number of pool stars of (pixel, half): inversion on word 0 of Philox(p, 2^32 - 1, set, LO|h)
 * below 10, transformed rejection with point index 2^32 - 1 at and above (the total has its own
 * boundary: one draw per pixel and half). */
#define OR_POOL_TOTAL_LIMIT 10.0f
static uint32_t or_pool_total(const or_pool *pl, uint64_t seed, uint32_t pix, uint32_t set, uint32_t half,
                              int *err)
{
    if (pl->n == 0) return 0u;
    if (pl->lam < OR_POOL_TOTAL_LIMIT) {
        uint32_t w[4];
        or_call(seed, pix, 0xFFFFFFFFu, set, or_tag(OR_KIND_LO, half, 0), w);
        return or_poisson_inversion(pl->lam, w[0]);
    }
    float c6[6];
    or_ptrs_setup(pl->lam, c6);
    uint32_t n = or_poisson_ptrs(c6, seed, pix, 0xFFFFFFFFu, set, half, NULL);
    if (n == UINT32_MAX) { if (err) *err = 1; return 0u; }
    return n;
}

int or_simulate(int n_pts, int n_bands, const float *lam_h, const double *flux, int n_im,
                uint32_t pix_begin, uint32_t pix_end, uint32_t set, uint64_t seed, int dust,
                double log_ebv, double dust_sigma, const double *r_ext, double *image,
                uint32_t *counts, int n_threads, int pool)
{
    int err = 0;
    size_t npix = (size_t)n_im * (size_t)n_im;
    or_pool pools[2];
    if (pool)
        for (int h = 0; h < 2; ++h) or_pool_build(lam_h + (size_t)h * n_pts, n_pts, &pools[h]);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16) reduction(| : err)
#endif
    for (long long pl = (long long)pix_begin; pl < (long long)pix_end; ++pl) {
        uint32_t p = (uint32_t)pl;
        double F[2][8];
        memset(F, 0, sizeof F);
        for (uint32_t h = 0; h < 2; ++h) {
            for (uint32_t i = 0; i < (uint32_t)n_pts; ++i) {
                float lam = lam_h[(size_t)h * n_pts + i];
                if (pool && lam < OR_INV_LIMIT) continue;      /* drawn through the pool below */
                int e = 0;
                uint32_t n = or_draw(lam, seed, p, i, set, h, &e);
                err |= e;
                if (counts) counts[(size_t)(p - pix_begin) * 2u * n_pts + h * n_pts + i] = n;
                if (n == 0u) continue;
                for (int b = 0; b < n_bands; ++b) F[h][b] += (double)n * flux[(size_t)i * n_bands + b];
            }
            if (!pool) continue;
            if (counts)
                for (uint32_t j = 0; j < pools[h].n; ++j)
                    counts[(size_t)(p - pix_begin) * 2u * n_pts + h * n_pts + pools[h].idx[j]] = 0u;
            int e = 0;
            uint32_t n_star = or_pool_total(&pools[h], seed, p, set, h, &e);
            err |= e;
            uint32_t w[4];
            for (uint32_t st = 0; st < n_star; ++st) {
                if ((st & 3u) == 0u)
                    or_call(seed, p, 0x80000000u | (st >> 2), set, or_tag(OR_KIND_HI, h, 0), w);
                uint32_t i = or_pool_pick(&pools[h], w[st & 3u]);
                if (counts) counts[(size_t)(p - pix_begin) * 2u * n_pts + h * n_pts + i] += 1u;
                for (int b = 0; b < n_bands; ++b) F[h][b] += flux[(size_t)i * n_bands + b];
            }
        }
        double fac[8];
        if (dust) or_dust_factors(seed, p, set, n_bands, log_ebv, dust_sigma, r_ext, fac);
        for (int b = 0; b < n_bands; ++b) {
            double v = F[0][b] + (dust ? fac[b] * F[1][b] : F[1][b]);
            if (image) image[(size_t)b * npix + p] = v;
        }
    }
    if (pool)
        for (int h = 0; h < 2; ++h) { free(pools[h].idx); free(pools[h].thr); }
    (void)n_threads;
    return err;
}

/* ------------------------------------------------------------------------------------- */
/* PSF, noise, magnitudes, Hess diagram (Section 2.1 Panels E-F, Section 2.5)             */
/* ------------------------------------------------------------------------------------- */

/* Periodic convolution, FP64: out[y][x] = sum_{u,v} K[u][v] in[(y+R-u) mod N][(x+R-v) mod N]. */
void or_psf(int n_im, int ksize, const float *kernel, const double *in, double *out)
{
    int R = ksize / 2;
    for (int y = 0; y < n_im; ++y)
        for (int x = 0; x < n_im; ++x) {
            double s = 0.0;
            for (int u = 0; u < ksize; ++u) {
                int yy = ((y + R - u) % n_im + n_im) % n_im;
                for (int v = 0; v < ksize; ++v) {
                    int xx = ((x + R - v) % n_im + n_im) % n_im;
                    s += (double)kernel[u * ksize + v] * in[(size_t)yy * n_im + xx];
                }
            }
            out[(size_t)y * n_im + x] = s;
        }
}

/* Sub-pixel PSFs (Section 2.2): the image is a 4x4 grid of regions; output pixel (y, x) belongs to
 * region (4y/n, 4x/n) (integer division) and is convolved (periodically) with that region's
 * kernel, kernels[(4 ry + rx) * ksize^2 ..]. */
void or_psf_grid(int n_im, int ksize, const float *kernels, const double *in, double *out)
{
    int R = ksize / 2;
    for (int y = 0; y < n_im; ++y)
        for (int x = 0; x < n_im; ++x) {
            const float *kernel = kernels + (size_t)((4 * y / n_im) * 4 + 4 * x / n_im) * ksize * ksize;
            double s = 0.0;
            for (int u = 0; u < ksize; ++u) {
                int yy = ((y + R - u) % n_im + n_im) % n_im;
                for (int v = 0; v < ksize; ++v) {
                    int xx = ((x + R - v) % n_im + n_im) % n_im;
                    s += (double)kernel[u * ksize + v] * in[(size_t)yy * n_im + xx];
                }
            }
            out[(size_t)y * n_im + x] = s;
        }
}

/* Photon and sky noise (noise = sqrt(counts), sky subtracted in expectation) and magnitudes.
 * F' = F + sqrt(max(F + sky, 0)) z_b, z from Box-Muller of the pixel's NOISE call for band pair
 * b >> 1 (cos for even b, sin for odd b).  m_b = ZP_b - 2.5 log10(F'_b / t_b) in FP64, rounded
 * to FP32.  A pixel is valid when F'_0 > 0 and F'_1 > 0.  mag = m_0, colour = m_1 - m_0 (FP32). */
void or_noise_mags(int n_im, int n_bands, const double *image, int noise, const double *sky,
                   const double *zp, const double *exptime, uint32_t set, uint64_t seed,
                   float *mag, float *colour, uint8_t *valid, double *fluxes_out)
{
    size_t npix = (size_t)n_im * (size_t)n_im;
    for (size_t p = 0; p < npix; ++p) {
        double Fp[8];
        for (int b = 0; b < n_bands; ++b) {
            double F = image[(size_t)b * npix + p];
            if (noise) {
                uint32_t w[4];
                or_call(seed, (uint32_t)p, (uint32_t)(b >> 1), set, or_tag(OR_KIND_NOISE, 0, 0), w);
                double u1 = (double)or_uniform(w[0]), u2 = (double)or_uniform(w[1]);
                double r = sqrt(-2.0 * log(u1));
                double z = (b & 1) ? r * sin(2.0 * M_PI * u2) : r * cos(2.0 * M_PI * u2);
                double var = F + sky[b];
                if (var < 0.0) var = 0.0;
                F = F + sqrt(var) * z;
            }
            Fp[b] = F;
            if (fluxes_out) fluxes_out[(size_t)b * npix + p] = F;
        }
        int ok = Fp[0] > 0.0 && Fp[1] > 0.0;
        valid[p] = (uint8_t)ok;
        if (!ok) { mag[p] = 0.0f; colour[p] = 0.0f; continue; }
        float m0 = (float)(zp[0] - 2.5 * log10(Fp[0] / exptime[0]));
        float m1 = (float)(zp[1] - 2.5 * log10(Fp[1] / exptime[1]));
        mag[p] = m0;
        colour[p] = m1 - m0;
    }
}

/* Hess diagram with the FP32 bin rule ix = floor((colour - c_lo) * inv_w), iy likewise for the
 * magnitude; hist[iy][ix].  counters[0] = valid pixels outside the grid, counters[1] = invalid
 * pixels.  moments = {sum colour, sum mag, n_valid} over valid pixels, FP64. */
void or_hess(size_t n, const float *mag, const float *colour, const uint8_t *valid, int nx,
             int ny, double c_lo, double m_lo, double width, uint32_t *hist, uint32_t *counters,
             double *moments)
{
    const float c_lo_f = (float)c_lo, m_lo_f = (float)m_lo, inv_w = (float)(1.0 / width);
    memset(hist, 0, sizeof(uint32_t) * (size_t)nx * ny);
    counters[0] = counters[1] = 0;
    moments[0] = moments[1] = moments[2] = 0.0;
    for (size_t p = 0; p < n; ++p) {
        if (!valid[p]) { counters[1]++; continue; }
        moments[0] += (double)colour[p];
        moments[1] += (double)mag[p];
        moments[2] += 1.0;
        float cx = colour[p] - c_lo_f;
        cx = cx * inv_w;
        float my = mag[p] - m_lo_f;
        my = my * inv_w;
        float fx = floorf(cx), fy = floorf(my);
        if (fx >= 0.0f && fx < (float)nx && fy >= 0.0f && fy < (float)ny)
            hist[(size_t)fy * nx + (size_t)fx]++;
        else
            counters[0]++;
    }
}
