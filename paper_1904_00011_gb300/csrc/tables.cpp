// Host table builder of libpcmd (compiled with -ffp-contract=off: every FP64 operation below is
// one IEEE operation in the order written, so the FP32 tables are a fixed function of the
// parameters).
//
// Weights (Section 2.1, Section 2.2): lambda_jki = SFH_j * MDF_k * IMF_jk,i with
//   SFH_j  = 10^log_sfh_j                          (S5, stars per pixel formed in bin j)
//   MDF_k  = exp(-((feh_k - mu)/sigma)^2 / 2) normalised over the grid, weights < mdf_cut
//            removed and renormalised (M2/M3); sigma <= 0 selects the nearest grid point
//   IMF_i  = integral of m^-slope over [e_i, e_i+1], e the geometric midpoints of the masses
//            (outer edges mirrored), normalised over the isochrone (Salpeter)
// Dust halves: (1 - F) lambda in front, F lambda behind the screen (thin screen, F_dust).
// Inversion thresholds: with p_0 = e^-lambda, p_k = p_{k-1} lambda / k, F_k = sum p, the draw
// word x gives n > k iff x > Z_k = ceil(F_k 2^32 - 1/2) - 1 (saturating at 2^32 - 1).
#include "tables.h"

#include <cmath>
#include <cstring>

namespace pcmd {

static inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

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

void Model::lambdas(const pcmd_params &p, std::vector<float> (&lam_h)[2]) const {
    std::vector<double> mdf;
    mdf_weights(p.feh_mean, p.feh_sigma, mdf);
    const size_t P = (size_t)n_points();
    lam_h[0].assign(P, 0.0f);
    lam_h[1].assign(P, 0.0f);
    for (int j = 0; j < n_ages; ++j) {
        const double sfh = std::pow(10.0, p.log_sfh[j]);
        for (int k = 0; k < n_feh; ++k) {
            const double wjk = sfh * mdf[k];
            const size_t base = ((size_t)j * n_feh + k) * n_mass;
            for (int i = 0; i < n_mass; ++i) {
                const double lam = wjk * imf[base + i];
                double l0, l1;
                if (!dust || f_dust <= 0.0) {
                    l0 = lam;
                    l1 = 0.0;
                } else if (f_dust >= 1.0) {
                    l0 = 0.0;
                    l1 = lam;
                } else {
                    l0 = lam * (1.0 - f_dust);
                    l1 = lam * f_dust;
                }
                lam_h[0][base + i] = (float)l0;
                lam_h[1][base + i] = (float)l1;
            }
        }
    }
}

void Model::fluxes(double dmod, std::vector<float> &flux) const {
    const size_t P = (size_t)n_points();
    flux.assign(P * n_bands, 0.0f);
    for (size_t i = 0; i < P; ++i)
        for (int b = 0; b < n_bands; ++b) {
            double s = abs_mag[i * n_bands + b] + dmod;
            s = s - zeropoint[b];
            s = -0.4 * s;
            const double f = std::pow(10.0, s);
            flux[i * n_bands + b] = (float)(exptime[b] * f);
        }
}

uint32_t threshold_of(double F) {
    const double T = std::ceil(std::ldexp(F, 32) - 0.5);
    if (T >= 4294967296.0) return 0xFFFFFFFFu;
    return (uint32_t)(T - 1.0);
}

int inversion_thresholds(float lam_f, uint32_t *z, int cap) {
    const double lam = (double)lam_f;
    double p = std::exp(-lam);
    double F = p;
    int n = 0;
    z[n++] = threshold_of(F);
    if (z[0] == 0xFFFFFFFFu) return n;
    for (int k = 1; k < cap; ++k) {
        p = p * lam;
        p = p / (double)k;
        F = F + p;
        const uint32_t t = threshold_of(F);
        z[n++] = t;
        if (t == 0xFFFFFFFFu) break;
    }
    return n;
}

void ptrs_constants(float lam_f, PtrsRec &r) {
    const double lam = (double)lam_f;
    const double slam = std::sqrt(lam);
    const double b = 0.931 + 2.53 * slam;
    const double a = -0.059 + 0.02483 * b;
    const double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
    const double vr = 0.9277 - 3.6224 / (b - 2.0);
    r.lam = lam_f;
    r.b = (float)b;
    r.a = (float)a;
    r.twoa = (float)(2.0 * a);
    r.vr = (float)vr;
    r.log_ia = (float)std::log(inv_alpha);
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

// Device table of one model, appended to `buf` (16-byte aligned sections).
void build_set_tables(const Model &m, const pcmd_params &p, std::vector<uint8_t> &buf,
                      SetDesc &d, SetStats &st) {
    std::vector<float> lam_h[2];
    std::vector<float> flux;
    m.lambdas(p, lam_h);
    m.fluxes(p.dmod, flux);
    const int B = m.n_bands;
    const uint32_t P = (uint32_t)m.n_points();
    const uint32_t G = (P + 7) / 8;
    const uint32_t rec = group_rec_bytes(B);
    const size_t base = align16(buf.size());

    std::vector<uint8_t> grp[2];
    std::vector<SlowRec> slow[2];
    std::vector<PtrsRec> ptrs[2];
    std::vector<uint32_t> tail;
    uint32_t z[kInvCap];
    st = SetStats();
    for (int h = 0; h < 2; ++h) {
        slow[h].assign((size_t)G * 8, SlowRec{0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u});
        for (uint32_t g = 0; g < G; ++g) {
            uint16_t zc0[8], zc1[8];
            float fl[8][kMaxBands];
            bool active = false;
            for (uint32_t j = 0; j < 8; ++j) {
                const uint32_t i = g * 8 + j;
                zc0[j] = 0xFFFFu;
                zc1[j] = 0xFFFFu;
                for (int b = 0; b < kMaxBands; ++b) fl[j][b] = 0.0f;
                if (i >= P) continue;
                for (int b = 0; b < B; ++b) fl[j][b] = flux[(size_t)i * B + b];
                const float lam = lam_h[h][i];
                if (!(lam > 0.0f)) continue;
                if (lam >= kPtrsThreshold) {
                    PtrsRec r;
                    std::memset(&r, 0, sizeof r);
                    r.i = i;
                    ptrs_constants(lam, r);
                    for (int b = 0; b < B; ++b) r.flux[b] = flux[(size_t)i * B + b];
                    ptrs[h].push_back(r);
                    continue;
                }
                const int nz = inversion_thresholds(lam, z, kInvCap);
                if (z[0] == 0xFFFFFFFFu) continue;
                SlowRec &s = slow[h][i];
                s.z0 = z[0];
                s.z1 = nz > 1 ? z[1] : 0xFFFFFFFFu;
                s.tail_off = (uint32_t)tail.size();
                s.tail_len = 0;
                for (int k = 2; k < nz; ++k) {
                    if (z[k] == 0xFFFFFFFFu) break;
                    tail.push_back(z[k]);
                    s.tail_len++;
                }
                zc0[j] = (uint16_t)(s.z0 >> 16);
                zc1[j] = (uint16_t)(s.z1 >> 16);
                active = true;
            }
            if (!active) continue;
            const size_t o = grp[h].size();
            grp[h].resize(o + rec, 0);
            uint8_t *r = grp[h].data() + o;
            std::memcpy(r, &g, 4);
            std::memcpy(r + 16, zc0, 16);
            std::memcpy(r + 32, zc1, 16);
            for (uint32_t j = 0; j < 8; ++j) std::memcpy(r + 48 + j * B * 4, fl[j], (size_t)B * 4);
        }
        st.n_inv_groups[h] = (uint32_t)(grp[h].size() / rec);
        st.n_ptrs[h] = (uint32_t)ptrs[h].size();
    }
    if (tail.empty()) tail.push_back(0xFFFFFFFFu);

    size_t off = base;
    auto place = [&](size_t bytes) {
        const size_t o = off;
        off = align16(off + bytes);
        return o;
    };
    for (int h = 0; h < 2; ++h) {
        d.grp_off[h] = place(grp[h].size());
        d.slow_off[h] = place(slow[h].size() * sizeof(SlowRec));
        d.ptrs_off[h] = place(ptrs[h].size() * sizeof(PtrsRec));
        d.n_grp[h] = st.n_inv_groups[h];
        d.n_ptrs[h] = st.n_ptrs[h];
    }
    d.tail_off = place(tail.size() * 4);
    buf.resize(off, 0);
    for (int h = 0; h < 2; ++h) {
        if (!grp[h].empty()) std::memcpy(buf.data() + d.grp_off[h], grp[h].data(), grp[h].size());
        std::memcpy(buf.data() + d.slow_off[h], slow[h].data(), slow[h].size() * sizeof(SlowRec));
        if (!ptrs[h].empty())
            std::memcpy(buf.data() + d.ptrs_off[h], ptrs[h].data(), ptrs[h].size() * sizeof(PtrsRec));
    }
    std::memcpy(buf.data() + d.tail_off, tail.data(), tail.size() * 4);

    // dust screen of this model (Section 2.2): E = 10^log_ebv exp(sigma z)
    d.dust_on = m.dust ? 1u : 0u;
    d.dust_a = (float)(std::log(10.0) * p.log_ebv);
    d.dust_sigma = (float)p.dust_sigma;
    for (int b = 0; b < kMaxBands; ++b) d.dust_c[b] = b < B ? (float)(-0.4 * m.r_ext[b]) : 0.0f;
    st.cost_per_pixel = 60.0 * (st.n_inv_groups[0] + st.n_inv_groups[1]) +
                        180.0 * (st.n_ptrs[0] + st.n_ptrs[1]) + 200.0;
}

}  // namespace pcmd
