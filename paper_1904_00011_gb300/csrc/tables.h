// Host-side model and table builder of libpcmd.
#pragma once
#include <stdint.h>
#include <functional>
#include <vector>

#include "../../include/pcmd.h"
#include "pcmd_internal.h"

namespace pcmd {

// Parameter-independent part of a context: isochrones, instrument constants, IMF weights.
struct Model {
    int n_bands = 2, n_ages = 1, n_feh = 1, n_mass = 1;
    std::vector<double> feh, mass, abs_mag;
    std::vector<double> imf;   // [n_ages][n_feh][n_mass], each isochrone sums to 1
    std::vector<double> base_flux;  // [P][n_bands] electrons per star at distance modulus 0
    double imf_slope = 2.35, mdf_cut = 0.01, f_dust = 0.5;
    double exptime[kMaxBands] = {1, 1, 1, 1}, zeropoint[kMaxBands] = {0, 0, 0, 0};
    double r_ext[kMaxBands] = {0, 0, 0, 0};
    bool dust = false;

    int n_points() const { return n_ages * n_feh * n_mass; }
    void build_imf();
    void build_base_flux();
    void mdf_weights(double mu, double sigma, std::vector<double> &w) const;
    void lambdas(const pcmd_params &p, std::vector<float> (&lam_h)[2]) const;
    void fluxes(double dmod, std::vector<float> &flux) const;
};

struct SetStats {
    uint32_t n_inv_groups[2] = {0, 0};
    uint32_t n_dense[2] = {0, 0};
    uint32_t n_ptrs[2] = {0, 0};
    double cost_per_pixel = 0.0;
};

uint32_t threshold_of(double F);
int inversion_thresholds(float lam, uint32_t *z, int cap);
void ptrs_constants(float lam, PtrsRec &r);
void stirlerr_table(float out[16]);
// Group records, transformed-rejection records and tail thresholds of a range of groups.
struct Part {
    std::vector<uint8_t> grp;
    std::vector<uint8_t> dense;
    std::vector<PtrsRec> ptrs;
    std::vector<uint32_t> tail;
};

// Host form of one model's device table.
struct SetTables {
    std::vector<float> lam_h[2], flux;
    std::vector<SlowRec> slow[2];
    std::vector<Part> parts[2];
    int n_parts = 1;
    uint32_t G = 0, rec = 0;
    size_t tail_total = 0;
    size_t bytes = 0;       // size of the emitted table
    SetDesc d;              // offsets relative to the table start
    SetStats st;
};

void build_set_tables(const Model &m, const pcmd_params &p, SetTables &t, bool parallel);
void emit_set_tables(const SetTables &t, uint8_t *dst);
void parallel_for(int n, const std::function<void(int)> &f);

}  // namespace pcmd
