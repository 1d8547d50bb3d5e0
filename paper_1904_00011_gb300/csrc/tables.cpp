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

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <mutex>
#include <thread>

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

void Model::fluxes(double dmod, std::vector<float> &flux) const {
    const size_t n = base_flux.size();
    flux.resize(n);
    const double f = std::pow(10.0, -0.4 * dmod);
    for (size_t i = 0; i < n; ++i) flux[i] = (float)(base_flux[i] * f);
}

// Z = ceil(F 2^32 - 1/2) - 1 with F 2^32 - 1/2 exact in FP64 and non-negative (F >= e^-10):
// the ceiling is the truncation plus one unless the value is already an integer.
uint32_t threshold_of(double F) {
    const double y = F * 4294967296.0 - 0.5;
    if (y >= 4294967295.0) return 0xFFFFFFFFu;   // T = ceil(y) >= 2^32
    const uint64_t t = (uint64_t)y;
    const uint64_t T = t + (y > (double)t ? 1u : 0u);
    return (uint32_t)(T - 1u);
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

// ---------------------------------------------------------------------------------------
// Worker pool: run(n, f) calls f(0..n-1) on the pool's threads and the caller.
// ---------------------------------------------------------------------------------------
class Pool {
public:
    explicit Pool(int n_workers) {
        for (int t = 0; t < n_workers; ++t) th_.emplace_back([this] { loop(); });
    }
    ~Pool() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : th_) t.join();
    }
    int size() const { return (int)th_.size() + 1; }
    void run(int n, const std::function<void(int)> &f) {
        if (n <= 1 || th_.empty()) {
            for (int i = 0; i < n; ++i) f(i);
            return;
        }
        std::unique_lock<std::mutex> lk(mu_);
        job_ = &f;
        n_ = n;
        next_ = 0;
        left_ = n;
        ++gen_;
        lk.unlock();
        cv_.notify_all();
        work();
        lk.lock();
        done_.wait(lk, [this] { return left_ == 0; });
        job_ = nullptr;
    }

private:
    void work() {
        while (true) {
            int i;
            const std::function<void(int)> *f;
            {
                std::lock_guard<std::mutex> g(mu_);
                if (!job_ || next_ >= n_) return;
                i = next_++;
                f = job_;
            }
            (*f)(i);
            std::lock_guard<std::mutex> g(mu_);
            if (--left_ == 0) done_.notify_all();
        }
    }
    void loop() {
        uint64_t seen = 0;
        while (true) {
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || (gen_ != seen && job_ && next_ < n_); });
                if (stop_) return;
                seen = gen_;
            }
            work();
        }
    }
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_, done_;
    const std::function<void(int)> *job_ = nullptr;
    int n_ = 0, next_ = 0, left_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};

static Pool &pool() {
    static Pool p([] {
        const unsigned hc = std::thread::hardware_concurrency();
        return (int)std::min(15u, hc > 1 ? hc - 1 : 0u);
    }());
    return p;
}

void parallel_for(int n, const std::function<void(int)> &f) { pool().run(n, f); }

static void build_part(const Model &m, const std::vector<float> &lam, const std::vector<float> &flux,
                       uint32_t g0, uint32_t g1, SlowRec *slow, Part &out) {
    const int B = m.n_bands;
    const uint32_t P = (uint32_t)m.n_points();
    const uint32_t rec = group_rec_bytes(B);
    uint32_t z[kInvCap];
    out.grp.clear();
    out.dense.clear();
    out.ptrs.clear();
    out.tail.clear();
    out.grp.reserve((size_t)(g1 - g0) * rec);
    for (uint32_t g = g0; g < g1; ++g) {
        uint16_t zc0[8], zc1[8];
        float fl[8][kMaxBands];
        bool active = false;
        float max_lam = 0.0f;
        for (uint32_t j = 0; j < 8; ++j) {
            const uint32_t i = g * 8 + j;
            zc0[j] = 0xFFFFu;
            zc1[j] = 0xFFFFu;
            for (int b = 0; b < kMaxBands; ++b) fl[j][b] = 0.0f;
            SlowRec &sr = slow[(size_t)g * 8 + j];
            sr = SlowRec{0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u};
            if (i >= P) continue;
            for (int b = 0; b < B; ++b) fl[j][b] = flux[(size_t)i * B + b];
            const float l = lam[i];
            if (!(l > 0.0f)) continue;
            if (l >= kPtrsThreshold) {
                PtrsRec r;
                std::memset(&r, 0, sizeof r);
                r.i = i;
                ptrs_constants(l, r);
                for (int b = 0; b < B; ++b) r.flux[b] = flux[(size_t)i * B + b];
                out.ptrs.push_back(r);
                continue;
            }
            const int nz = inversion_thresholds(l, z, kInvCap);
            if (z[0] == 0xFFFFFFFFu) continue;
            sr.z0 = z[0];
            sr.z1 = nz > 1 ? z[1] : 0xFFFFFFFFu;
            sr.tail_off = (uint32_t)out.tail.size();   // local; rebased when parts are joined
            for (int k = 2; k < nz; ++k) {
                if (z[k] == 0xFFFFFFFFu) break;
                out.tail.push_back(z[k]);
                sr.tail_len++;
            }
            // search start near lambda for the device's threshold walk: 2 <= ks <= len + 1
            const uint32_t len = sr.tail_len;
            uint32_t ks = (uint32_t)l;
            if (ks > len + 1u) ks = len + 1u;
            if (ks < 2u) ks = 2u;
            sr.tail_len = len | (ks << 16);
            zc0[j] = (uint16_t)(sr.z0 >> 16);
            zc1[j] = (uint16_t)(sr.z1 >> 16);
            active = true;
            if (l > max_lam) max_lam = l;
        }
        if (!active) continue;
        std::vector<uint8_t> &dst = max_lam >= kDenseLam ? out.dense : out.grp;
        const size_t o = dst.size();
        dst.resize(o + rec, 0);
        uint8_t *r = dst.data() + o;
        uint32_t zs[8];
        for (uint32_t j = 0; j < 8; ++j) zs[j] = (uint32_t)zc0[j] << 16;
        std::memcpy(r, &g, 4);
        std::memcpy(r + kRecZs, zs, 32);
        std::memcpy(r + kRecZc1, zc1, 16);
        for (uint32_t j = 0; j < 8; ++j) std::memcpy(r + kRecFlux + j * B * 4, fl[j], (size_t)B * 4);
    }
}

// Tables of one model, built over the worker pool when `parallel` is set (large grids).
// Offsets in `t.d` are relative to the start of the model's table; emit_set_tables writes it.
void build_set_tables(const Model &m, const pcmd_params &p, SetTables &t, bool parallel) {
    m.lambdas(p, t.lam_h);
    m.fluxes(p.dmod, t.flux);
    const int B = m.n_bands;
    const uint32_t P = (uint32_t)m.n_points();
    const uint32_t G = (P + 7) / 8;
    const uint32_t rec = group_rec_bytes(B);
    int n_parts = 1;
    if (parallel && G >= 256) n_parts = std::min<int>(pool().size() * 2, (int)(G / 64));
    t.n_parts = n_parts;
    t.G = G;
    t.rec = rec;
    for (int h = 0; h < 2; ++h) {
        t.slow[h].resize((size_t)G * 8);
        t.parts[h].resize(n_parts);
    }
    auto task = [&](int q) {
        const int h = q / n_parts, k = q % n_parts;
        const uint32_t g0 = (uint32_t)((uint64_t)G * k / n_parts);
        const uint32_t g1 = (uint32_t)((uint64_t)G * (k + 1) / n_parts);
        build_part(m, t.lam_h[h], t.flux, g0, g1, t.slow[h].data(), t.parts[h][k]);
    };
    if (n_parts > 1) parallel_for(2 * n_parts, task);
    else for (int q = 0; q < 2; ++q) task(q);

    SetStats &st = t.st;
    SetDesc &d = t.d;
    st = SetStats();
    t.tail_total = 0;
    for (int h = 0; h < 2; ++h) {
        size_t ng = 0, np = 0, nd = 0;
        for (int k = 0; k < n_parts; ++k) {
            const uint32_t g0 = (uint32_t)((uint64_t)G * k / n_parts);
            const uint32_t g1 = (uint32_t)((uint64_t)G * (k + 1) / n_parts);
            const uint32_t base = (uint32_t)t.tail_total;
            if (base)
                for (size_t i = (size_t)g0 * 8; i < (size_t)g1 * 8; ++i)
                    if (t.slow[h][i].tail_len & 0xFFFFu) t.slow[h][i].tail_off += base;
            t.tail_total += t.parts[h][k].tail.size();
            ng += t.parts[h][k].grp.size() / rec;
            nd += t.parts[h][k].dense.size() / rec;
            np += t.parts[h][k].ptrs.size();
        }
        st.n_inv_groups[h] = (uint32_t)ng;
        st.n_dense[h] = (uint32_t)nd;
        st.n_ptrs[h] = (uint32_t)np;
    }
    size_t off = 0;
    auto place = [&](size_t bytes) {
        const size_t o = off;
        off = align16(off + bytes);
        return o;
    };
    for (int h = 0; h < 2; ++h) {
        d.grp_off[h] = place((size_t)st.n_inv_groups[h] * rec);
        d.dense_off[h] = place((size_t)st.n_dense[h] * rec);
        d.n_dense[h] = st.n_dense[h];
        d.slow_off[h] = place(t.slow[h].size() * sizeof(SlowRec));
        d.ptrs_off[h] = place((size_t)st.n_ptrs[h] * sizeof(PtrsRec));
        d.n_grp[h] = st.n_inv_groups[h];
        d.n_ptrs[h] = st.n_ptrs[h];
    }
    d.tail_off = place(std::max<size_t>(t.tail_total, 1) * 4);
    t.bytes = off;

    // dust screen of this model (Section 2.2): E = 10^log_ebv exp(sigma z)
    d.dust_on = m.dust ? 1u : 0u;
    d.dust_a = (float)(std::log(10.0) * p.log_ebv);
    d.dust_sigma = (float)p.dust_sigma;
    for (int b = 0; b < kMaxBands; ++b) d.dust_c[b] = b < B ? (float)(-0.4 * m.r_ext[b]) : 0.0f;
    st.cost_per_pixel = 60.0 * (st.n_inv_groups[0] + st.n_inv_groups[1]) +
                        400.0 * (st.n_dense[0] + st.n_dense[1]) +
                        180.0 * (st.n_ptrs[0] + st.n_ptrs[1]) + 200.0;
}

// Write the model's table (t.bytes bytes) at dst.
void emit_set_tables(const SetTables &t, uint8_t *dst) {
    const SetDesc &d = t.d;
    for (int h = 0; h < 2; ++h) {
        size_t go = d.grp_off[h], po = d.ptrs_off[h], dd = d.dense_off[h];
        for (int k = 0; k < t.n_parts; ++k) {
            const Part &pt = t.parts[h][k];
            if (!pt.grp.empty()) std::memcpy(dst + go, pt.grp.data(), pt.grp.size());
            go += pt.grp.size();
            if (!pt.dense.empty()) std::memcpy(dst + dd, pt.dense.data(), pt.dense.size());
            dd += pt.dense.size();
            if (!pt.ptrs.empty()) std::memcpy(dst + po, pt.ptrs.data(), pt.ptrs.size() * sizeof(PtrsRec));
            po += pt.ptrs.size() * sizeof(PtrsRec);
        }
        std::memcpy(dst + d.slow_off[h], t.slow[h].data(), t.slow[h].size() * sizeof(SlowRec));
    }
    uint32_t *tail = reinterpret_cast<uint32_t *>(dst + d.tail_off);
    size_t o = 0;
    for (int h = 0; h < 2; ++h)
        for (int k = 0; k < t.n_parts; ++k) {
            const Part &pt = t.parts[h][k];
            if (!pt.tail.empty()) std::memcpy(tail + o, pt.tail.data(), pt.tail.size() * 4);
            o += pt.tail.size();
        }
    if (o == 0) tail[0] = 0xFFFFFFFFu;
}

}  // namespace pcmd
