// Host part of the model of libpcmd (compiled with -ffp-contract=off: every FP64 operation below
// is one IEEE operation in the order written).  The per-point tables are built on the device
// (tables_dev.cu) from the per-isochrone weights and the arrays computed here.
//
// Weights (Section 2.1, Section 2.2): lambda_jki = SFH_j * MDF_k * IMF_jk,i with
//   SFH_j  = 10^log_sfh_j                          (S5, stars per pixel formed in bin j)
//   MDF_k  = exp(-((feh_k - mu)/sigma)^2 / 2) normalised over the grid, weights < mdf_cut
//            removed and renormalised (M2/M3); sigma <= 0 is M1: one [Fe/H], the isochrone
//            interpolated between the two grid isochrones around it (m1_isochrone)
//   IMF_i  = integral of m^-slope over [e_i, e_i+1], e the geometric midpoints of the masses
//            (outer edges mirrored), normalised over the isochrone (Salpeter)
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace pcmd {

// Kroupa (2001) IMF integrated over [a, b]: xi(m) = k_s m^-alpha_s on the segments
// [0, 0.08), [0.08, 0.5), [0.5, inf) with alpha = 0.3, 1.3, 2.3 and k = 1, 0.08, 0.04 (continuous).
static double kroupa_cell(double a, double b) {
    const double lo[3] = {0.0, 0.08, 0.5}, hi[3] = {0.08, 0.5, 1.0e300};
    const double alpha[3] = {0.3, 1.3, 2.3}, k[3] = {1.0, 0.08, 0.04};
    double s = 0.0;
    for (int g = 0; g < 3; ++g) {
        const double x0 = a > lo[g] ? a : lo[g];
        const double x1 = b < hi[g] ? b : hi[g];
        if (x1 > x0) {
            const double e = 1.0 - alpha[g];
            double t = std::pow(x1, e) - std::pow(x0, e);
            t = t / e;
            s = s + k[g] * t;
        }
    }
    return s;
}

// IMF weights of one isochrone's mass points: the integral of the IMF over each point's cell
// (bounded by the geometric midpoints of neighbouring masses, outer edges mirrored),
// normalised over the isochrone.
static void imf_of_isochrone(const double *m, int n_mass, double slope, int kind, double *out) {
    if (n_mass == 1) {
        out[0] = 1.0;
        return;
    }
    std::vector<double> omega(n_mass), edge(n_mass + 1);
    for (int i = 1; i < n_mass; ++i) edge[i] = std::sqrt(m[i - 1] * m[i]);
    edge[0] = m[0] * m[0] / edge[1];
    edge[n_mass] = m[n_mass - 1] * m[n_mass - 1] / edge[n_mass - 1];
    const double a1 = 1.0 - slope;
    double s = 0.0;
    for (int i = 0; i < n_mass; ++i) {
        double w;
        if (kind == PCMD_IMF_KROUPA) {
            w = kroupa_cell(edge[i], edge[i + 1]);
        } else if (a1 != 0.0) {
            w = std::pow(edge[i + 1], a1) - std::pow(edge[i], a1);
            w = w / a1;
        } else {
            w = std::log(edge[i + 1] / edge[i]);
        }
        omega[i] = w;
        s = s + w;
    }
    for (int i = 0; i < n_mass; ++i) out[i] = omega[i] / s;
}

void Model::build_imf() {
    imf.assign((size_t)n_ages * n_feh * n_mass, 0.0);
    imf_max.assign((size_t)n_ages * n_feh, 0.0);
    for (int j = 0; j < n_ages; ++j)
        for (int k = 0; k < n_feh; ++k) {
            const size_t o = ((size_t)j * n_feh + k) * n_mass;
            imf_of_isochrone(&mass[o], n_mass, imf_slope, imf_kind, &imf[o]);
            for (int i = 0; i < n_mass; ++i) imf_max[(size_t)j * n_feh + k] = std::max(imf_max[(size_t)j * n_feh + k], imf[o + i]);
        }
    imf_desc = imf;
    for (size_t o = 0; o < imf_desc.size(); o += (size_t)n_mass)
        std::sort(imf_desc.begin() + (long)o, imf_desc.begin() + (long)o + n_mass, std::greater<double>());
}

void Model::mdf_weights(double mu, double sigma, std::vector<double> &w) const {
    w.assign(n_feh, 0.0);
    if (sigma > 0.0) {
        double s = 0.0;
        for (int k = 0; k < n_feh; ++k) {
            double t = feh[k] - mu;
            t = t / sigma;
            w[k] = std::exp(-0.5 * (t * t));
            s = s + w[k];
        }
        double s2 = 0.0;
        for (int k = 0; k < n_feh; ++k) {
            w[k] = w[k] / s;
            if (w[k] < mdf_cut) w[k] = 0.0;
            s2 = s2 + w[k];
        }
        for (int k = 0; k < n_feh; ++k) w[k] = w[k] / s2;
    } else {
        double t;
        w[m1_bracket(mu, t)] = 1.0;
    }
}

// M1 (Section 2.2): the grid isochrone k at or below mu and the fraction t in [0, 1) of the way
// to isochrone k + 1; mu outside the grid takes the end isochrone (t = 0).
int Model::m1_bracket(double mu, double &t) const {
    t = 0.0;
    if (n_feh == 1 || mu <= feh[0]) return 0;
    if (mu >= feh[n_feh - 1]) return n_feh - 1;
    int k = 0;
    while (k + 2 < n_feh && feh[k + 1] <= mu) ++k;
    t = (mu - feh[k]) / (feh[k + 1] - feh[k]);
    return k;
}

// The isochrones of [Fe/H] = feh_k + t (feh_k+1 - feh_k), one per age: every mass point's
// initial mass and absolute magnitudes interpolated linearly in [Fe/H] between the same mass
// point of the two grid isochrones, then the IMF weights and the electrons per star of those
// points.  imf_out[n_ages][n_mass], bflux_out[n_ages][n_mass][n_bands].
void Model::m1_isochrone(int k, double t, double *imf_out, double *bflux_out) const {
    std::vector<double> mi(n_mass);
    const double u = 1.0 - t;
    for (int j = 0; j < n_ages; ++j) {
        const size_t o0 = ((size_t)j * n_feh + k) * n_mass, o1 = o0 + n_mass;
        for (int i = 0; i < n_mass; ++i) mi[i] = u * mass[o0 + i] + t * mass[o1 + i];
        imf_of_isochrone(mi.data(), n_mass, imf_slope, imf_kind, imf_out + (size_t)j * n_mass);
        for (int i = 0; i < n_mass; ++i)
            for (int b = 0; b < n_bands; ++b) {
                const double mag = u * abs_mag[(o0 + i) * n_bands + b] + t * abs_mag[(o1 + i) * n_bands + b];
                bflux_out[((size_t)j * n_mass + i) * n_bands + b] = electrons_per_star(mag, b);
            }
    }
}

double Model::electrons_per_star(double mag, int b) const {
    double s = mag - zeropoint[b];
    s = -0.4 * s;
    return exptime[b] * std::pow(10.0, s);
}

// Electrons per star: t_b 10^(-0.4 (M_b + dmod - ZP_b)) = [t_b 10^(-0.4 (M_b - ZP_b))] 10^(-0.4 dmod);
// the bracket is computed once per context (base_flux), the distance factor once per model.
void Model::build_base_flux() {
    const size_t P = (size_t)n_points();
    base_flux.assign(P * n_bands, 0.0);
    for (size_t i = 0; i < P; ++i)
        for (int b = 0; b < n_bands; ++b) base_flux[i * n_bands + b] = electrons_per_star(abs_mag[i * n_bands + b], b);
}

void stirlerr_table(float out[16]) {
    out[0] = 0.0f;
    for (int k = 1; k < 16; ++k) {
        const double kd = (double)k;
        double s = std::lgamma(kd + 1.0);
        s = s - (kd + 0.5) * std::log(kd);
        s = s + kd;
        s = s - 0.5 * std::log(2.0 * M_PI);
        out[k] = (float)s;
    }
}

// Section 2.2 S1-S4.  Ages a in years, formation times t = T0 - a with T0 the oldest edge; the
// mass formed in bin [a_lo, a_hi) is the integral of the rate over t in [T0 - a_hi, T0 - a_lo].
bool sfh_bins(int model, const double *theta, int n_theta, int n_bins, const double *edges, double *out) {
    if (!theta || !edges || !out || n_bins < 1 || n_bins > PCMD_MAX_SFH || n_theta < 1) return false;
    for (int j = 0; j <= n_bins; ++j)
        if (!std::isfinite(edges[j]) || (j > 0 && !(edges[j] > edges[j - 1]))) return false;
    for (int i = 0; i < n_theta; ++i)
        if (!std::isfinite(theta[i])) return false;
    const double npix = std::pow(10.0, theta[0]);
    const double T0 = std::pow(10.0, edges[n_bins]);
    std::vector<double> m(n_bins, 0.0);
    if (model == PCMD_SFH_SSP) {
        if (n_theta < 2) return false;
        int j0 = -1;
        for (int j = 0; j < n_bins; ++j)
            if (theta[1] >= edges[j] && theta[1] < edges[j + 1]) j0 = j;
        if (j0 < 0) return false;
        m[j0] = 1.0;
    } else if (model == PCMD_SFH_CONSTANT) {
        for (int j = 0; j < n_bins; ++j) m[j] = std::pow(10.0, edges[j + 1]) - std::pow(10.0, edges[j]);
    } else if (model == PCMD_SFH_TAU || model == PCMD_SFH_DELAYED_TAU) {
        if (n_theta < 2 || !(theta[1] > 0.0)) return false;
        const double tau = theta[1] * 1.0e9;
        for (int j = 0; j < n_bins; ++j) {
            const double t1 = T0 - std::pow(10.0, edges[j + 1]);   // older edge: earlier time
            const double t2 = T0 - std::pow(10.0, edges[j]);
            const double e1 = std::exp(-t1 / tau), e2 = std::exp(-t2 / tau);
            if (model == PCMD_SFH_TAU) m[j] = tau * (e1 - e2);
            else m[j] = tau * (e1 * (t1 + tau) - e2 * (t2 + tau));
        }
    } else {
        return false;
    }
    double tot = 0.0;
    for (int j = 0; j < n_bins; ++j) tot += m[j];
    if (!(tot > 0.0)) return false;
    for (int j = 0; j < n_bins; ++j) {
        const double v = npix * (m[j] / tot);
        out[j] = v > 0.0 ? std::log10(v) : -30.0;
        if (out[j] < -30.0) out[j] = -30.0;
    }
    return true;
}

}  // namespace pcmd
