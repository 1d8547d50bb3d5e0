// Host part of the model of libpcmd (compiled with -ffp-contract=off: every FP64 operation below
// is one IEEE operation in the order written).  The per-point tables are built on the device
// (tables_dev.cu) from the per-isochrone weights and the arrays computed here.
//
// Weights (Section 2.1, Section 2.2): lambda_jki = SFH_j * MDF_k * IMF_jk,i with
//   SFH_j  = 10^log_sfh_j                          (S5, stars per pixel formed in bin j)
//   MDF_k  = exp(-((feh_k - mu)/sigma)^2 / 2) normalised over the grid, weights < mdf_cut
//            removed and renormalised (M2/M3); sigma <= 0 selects the nearest grid point
//   IMF_i  = integral of m^-slope over [e_i, e_i+1], e the geometric midpoints of the masses
//            (outer edges mirrored), normalised over the isochrone (Salpeter)
#include "tables.h"

#include <cmath>

namespace pcmd {

void Model::build_imf() {
    imf.assign((size_t)n_ages * n_feh * n_mass, 0.0);
    std::vector<double> omega(n_mass), edge(n_mass + 1);
    for (int j = 0; j < n_ages; ++j)
        for (int k = 0; k < n_feh; ++k) {
            const double *m = &mass[((size_t)j * n_feh + k) * n_mass];
            double s = 0.0;
            if (n_mass == 1) {
                omega[0] = 1.0;
                s = 1.0;
            } else {
                for (int i = 1; i < n_mass; ++i) edge[i] = std::sqrt(m[i - 1] * m[i]);
                edge[0] = m[0] * m[0] / edge[1];
                edge[n_mass] = m[n_mass - 1] * m[n_mass - 1] / edge[n_mass - 1];
                const double a1 = 1.0 - imf_slope;
                for (int i = 0; i < n_mass; ++i) {
                    double w;
                    if (a1 != 0.0) {
                        w = std::pow(edge[i + 1], a1) - std::pow(edge[i], a1);
                        w = w / a1;
                    } else {
                        w = std::log(edge[i + 1] / edge[i]);
                    }
                    omega[i] = w;
                    s = s + w;
                }
            }
            double *out = &imf[((size_t)j * n_feh + k) * n_mass];
            for (int i = 0; i < n_mass; ++i) out[i] = omega[i] / s;
        }
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
        int best = 0;
        for (int k = 1; k < n_feh; ++k)
            if (std::fabs(feh[k] - mu) < std::fabs(feh[best] - mu)) best = k;
        w[best] = 1.0;
    }
}


// Electrons per star: t_b 10^(-0.4 (M_b + dmod - ZP_b)) = [t_b 10^(-0.4 (M_b - ZP_b))] 10^(-0.4 dmod);
// the bracket is computed once per context (base_flux), the distance factor once per model.
void Model::build_base_flux() {
    const size_t P = (size_t)n_points();
    base_flux.assign(P * n_bands, 0.0);
    for (size_t i = 0; i < P; ++i)
        for (int b = 0; b < n_bands; ++b) {
            double s = abs_mag[i * n_bands + b] - zeropoint[b];
            s = -0.4 * s;
            base_flux[i * n_bands + b] = exptime[b] * std::pow(10.0, s);
        }
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

}  // namespace pcmd
