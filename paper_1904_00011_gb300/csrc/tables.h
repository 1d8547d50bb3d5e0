// Host-side model of libpcmd: parameter-independent arrays and the per-model MDF weights.
#pragma once
#include <stdint.h>
#include <vector>

#include "../../include/pcmd.h"
#include "pcmd_internal.h"

namespace pcmd {

// Parameter-independent part of a context: isochrones, instrument constants, IMF weights.
struct Model {
    int n_bands = 2, n_ages = 1, n_feh = 1, n_mass = 1;
    std::vector<double> feh, mass, abs_mag;
    std::vector<double> imf;   // [n_ages][n_feh][n_mass], each isochrone sums to 1
    std::vector<double> imf_max;   // [n_ages][n_feh] largest IMF weight of each isochrone
    std::vector<double> imf_desc;  // [n_ages][n_feh][n_mass] each isochrone's IMF weights, descending
    std::vector<double> base_flux;  // [P][n_bands] electrons per star at distance modulus 0
    double imf_slope = 2.35, mdf_cut = 0.01, f_dust = 0.5;
    double exptime[kMaxBands] = {1, 1, 1, 1}, zeropoint[kMaxBands] = {0, 0, 0, 0};
    double r_ext[kMaxBands] = {0, 0, 0, 0};
    bool dust = false;
    int imf_kind = 0;          // PCMD_IMF_POWER / PCMD_IMF_KROUPA

    int n_points() const { return n_ages * n_feh * n_mass; }
    void build_imf();
    void build_base_flux();
    double electrons_per_star(double mag, int band) const;
    void mdf_weights(double mu, double sigma, std::vector<double> &w) const;
    int m1_bracket(double mu, double &t) const;
    void m1_isochrone(int k, double t, double *imf_out, double *bflux_out) const;
};

void stirlerr_table(float out[16]);
// Parametric SFH on an age grid (PCMD_SFH_*): log10 stars per bin; false on bad input.
bool sfh_bins(int model, const double *theta, int n_theta, int n_bins, const double *edges, double *out);

}  // namespace pcmd
