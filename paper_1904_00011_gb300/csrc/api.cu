// C ABI of libpcmd (declared in include/pcmd.h): contexts, argument checks, table upload and
// the launch sequence of the forward model.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/pcmd.h"
#include "pcmd_internal.h"
#include "tables.h"
#include "tables_dev.h"

namespace pcmd {
}

using namespace pcmd;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    uint64_t gen = 0;       // bumped on every (re)allocation: contents of an older one are gone
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        ++gen;
        const size_t want = std::max<size_t>(bytes, 256);
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        ++gen;
    }
    template <class T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

struct HostBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap && p) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        const size_t want = std::max<size_t>(bytes, 256);
        cudaError_t e = cudaMallocHost(&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

}  // namespace

struct pcmd_ctx {
    pcmd_config cfg;
    Model model;
    std::vector<float> psf;     // [B][S][S]
    std::vector<float> psf25;   // [kMaxBands][625] when S == 25
    cudaStream_t st = nullptr;
    cudaStream_t cap_st = nullptr;
    int device = 0, n_sm = 1;
    int block = 256, split = 4, chunk = 256;   // launch shape (pcmd_set_launch; autotuned)
    uint32_t ptrs_cap = kPtrsMaxAttempts;   // transformed-rejection attempt cap of a draw

    SetDesc *desc_d = nullptr;  // the models' descriptors (inside tab_in, uploaded with it)
    DevBuf btab;                // word tables of the dense groups (allocated when needed)
    DevBuf tables, items, order, partials, part_begin, part_count, image, pix_off, hess,
        moments, counters, ll, psf_d, queue, err;
    DevBuf imf_d, bflux_d, tab_in, tab_scratch, insp;   // device table builder
    DevBuf ll_part, ll_ticket;                          // likelihood partials and per-set tickets
    HostBuf h_tab_in, h_items, h_order, h_meta, h_ll;
    cudaEvent_t staged = nullptr;
    bool staged_pending = false;
    TabLayout layout;
    std::vector<SetDesc> descs;
    std::vector<double> cost;
    std::vector<uint2> item_list;
    std::vector<uint32_t> order_list;

    int n_sets = 0;
    int draw_paths = kPathDense;    // draw paths the staged models can need (kPath* bits)
    std::vector<int> n_im;
    float *img_ptr = nullptr;
    bool have_images = false, have_hess = false;
    uint32_t *hess_ptr = nullptr;
    double *mom_ptr = nullptr;
    uint32_t *ctr_ptr = nullptr;

    // last content uploaded to small per-shape device arrays (the upload is skipped when equal)
    struct Uploaded {
        const void *dev = nullptr;
        uint64_t gen = 0;
        std::vector<uint8_t> bytes;
    };
    Uploaded up_items, up_order, up_part_begin, up_part_count, up_pix_off;

    // graph of the fused evaluation
    // instantiated graphs of the fused evaluation, one per shape (set count, work items, launch,
    // mock, and every device pointer the graph captured), least recently used evicted first:
    // a sampler loop over images of a few sizes replays without re-capturing
    struct GraphEntry {
        std::vector<size_t> key;
        cudaGraphExec_t exec = nullptr;
        uint64_t used = 0;
    };
    std::vector<GraphEntry> graphs;
    uint64_t graph_tick = 0;

    // kernel timing (pcmd_profile)
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[PCMD_KERNEL_KINDS];

    std::string err_text;
};

// Brackets one kernel launch with events on the context's stream while profiling is on.
struct KTimer {
    pcmd_ctx *ctx;
    int kind;
    cudaEvent_t a = nullptr, b = nullptr;
    KTimer(pcmd_ctx *c, int k, cudaStream_t st) : ctx(c), kind(k) {
        if (!ctx->profiling) return;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
    }
    void done(cudaStream_t st) {
        if (!a) return;
        cudaEventRecord(b, st);
        ctx->ev[kind].push_back({a, b});
        a = b = nullptr;
    }
};

#define CK(call)                                                                    \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ctx->err_text = std::string(#call) + ": " + cudaGetErrorString(e_);     \
            return e_ == cudaErrorMemoryAllocation ? PCMD_ERR_OOM : PCMD_ERR_CUDA;  \
        }                                                                           \
    } while (0)

// Asynchronous upload of a small per-shape array from pinned memory, skipped when the device
// buffer already holds exactly these bytes.
static cudaError_t upload_if_changed(pcmd_ctx::Uploaded &u, const DevBuf &dst, const void *src, size_t n,
                                     cudaStream_t st) {
    if (u.dev == dst.p && u.gen == dst.gen && u.bytes.size() == n && std::memcmp(u.bytes.data(), src, n) == 0)
        return cudaSuccess;
    const cudaError_t e = cudaMemcpyAsync(dst.p, src, n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        u.dev = dst.p;
        u.gen = dst.gen;
        u.bytes.assign(static_cast<const uint8_t *>(src), static_cast<const uint8_t *>(src) + n);
    } else {
        u.dev = nullptr;
    }
    return e;
}

static pcmd_status arg_error(pcmd_ctx *ctx, const std::string &why) {
    if (ctx) ctx->err_text = why;
    return PCMD_ERR_ARG;
}

static bool is_fin(double v) { return std::isfinite(v); }

static PixelConsts pixel_consts(const pcmd_ctx *ctx) {
    const pcmd_config &c = ctx->cfg;
    PixelConsts pc;
    std::memset(&pc, 0, sizeof pc);
    for (int b = 0; b < kMaxBands; ++b) {
        const bool on = b < c.n_bands;
        pc.sky[b] = on ? (float)c.sky[b] : 0.0f;
        pc.t[b] = on ? (float)c.exptime[b] : 1.0f;
        pc.zp[b] = on ? (float)c.zeropoint[b] : 0.0f;
        pc.zp_lo[b] = on ? (float)(c.zeropoint[b] - (double)pc.zp[b]) : 0.0f;
    }
    pc.c_lo = (float)c.hess_c_lo;
    pc.m_lo = (float)c.hess_m_lo;
    pc.inv_w = (float)(1.0 / c.hess_width);
    pc.nx = c.hess_nx;
    pc.ny = c.hess_ny;
    pc.noise = (c.flags & PCMD_FLAG_NOISE) ? 1 : 0;
    pc.seed = c.seed;
    return pc;
}

static pcmd_status check_params(pcmd_ctx *ctx, const pcmd_params *p, int n_sets, const int *n_im) {
    if (!p || !n_im) return arg_error(ctx, "params and n_im must not be NULL");
    if (n_sets < 1 || n_sets > ctx->cfg.max_sets) return arg_error(ctx, "n_sets outside 1..max_sets");
    for (int s = 0; s < n_sets; ++s) {
        if (n_im[s] < 1 || n_im[s] > ctx->cfg.max_im) return arg_error(ctx, "n_im outside 1..max_im");
        for (int j = 0; j < ctx->model.n_ages; ++j)
            if (!is_fin(p[s].log_sfh[j]) || p[s].log_sfh[j] > 7.0)
                return arg_error(ctx, "log_sfh must be finite and <= 7 (lambda must stay below 1e7)");
        if (!is_fin(p[s].feh_mean) || !is_fin(p[s].feh_sigma) || !is_fin(p[s].log_ebv) ||
            !is_fin(p[s].dust_sigma) || !is_fin(p[s].dmod))
            return arg_error(ctx, "non-finite parameter");
        if (p[s].dust_sigma < 0.0 || p[s].dust_sigma > 5.0) return arg_error(ctx, "dust_sigma outside [0, 5]");
        if (p[s].log_ebv > 2.0 || p[s].log_ebv < -20.0) return arg_error(ctx, "log_ebv outside [-20, 2]");
    }
    return PCMD_OK;
}

// Relative cost per pixel of a model, for the longest-first queue of a batch: lambda of every
// point from the same FP64 products as the device builder; groups with an inversion point,
// dense groups (a point at or above kDenseLam) and transformed-rejection points.
static double model_cost(const Model &m, const double *w, const double hf[2]) {
    // per isochrone: transformed-rejection points from the sorted IMF weights (binary search),
    // its groups counted as dense or sparse from its largest weight (an ordering estimate only)
    double c = 200.0;
    const double groups = (double)(m.n_mass + kGroup - 1) / (double)kGroup;
    for (int h = 0; h < 2; ++h) {
        if (hf[h] == 0.0) continue;
        for (int jk = 0; jk < m.n_ages * m.n_feh; ++jk) {
            const double s = w[jk] * hf[h];
            if (!(s > 0.0)) continue;
            const double *d = m.imf_desc.data() + (size_t)jk * m.n_mass;
            const double cut = (double)kPtrsThreshold / s;
            const long n_ptrs = std::upper_bound(d, d + m.n_mass, cut, std::greater<double>()) - d;
            c += 180.0 * (double)n_ptrs;
            c += groups * (s * m.imf_max[jk] >= (double)kDenseLam ? 700.0 : 70.0);
        }
    }
    return c;
}

static void half_factors(const Model &m, double hf[2]) {
    if (!m.dust || m.f_dust <= 0.0) {
        hf[0] = 1.0;
        hf[1] = 0.0;
    } else if (m.f_dust >= 1.0) {
        hf[0] = 0.0;
        hf[1] = 1.0;
    } else {
        hf[0] = 1.0 - m.f_dust;
        hf[1] = m.f_dust;
    }
}

// Stage n_sets models: the host computes the per-isochrone weights w_jk = SFH_j MDF_k and the
// distance factor of each model (FP64), one pinned upload carries them with the descriptors and
// the work items, and the device builds the tables (list lengths land in the descriptors).
// Items are pixel tiles of block / split pixels; `cost_sorted` orders the queue longest first.
static pcmd_status stage_sets(pcmd_ctx *ctx, const pcmd_params *p, int n_sets, const int *n_im,
                              uint32_t first_set_id, bool cost_sorted, int ppc,
                              float *insp_lam = nullptr, float *insp_flux = nullptr,
                              uint32_t *insp_z0 = nullptr) {
    const Model &m = ctx->model;
    const int B = m.n_bands;
    const uint32_t P = (uint32_t)m.n_points();
    const int nw = m.n_ages * m.n_feh;
    const TabLayout &L = ctx->layout;
    double hf[2];
    half_factors(m, hf);
    ctx->descs.assign(n_sets, SetDesc());
    ctx->cost.assign(n_sets, 0.0);
    ctx->item_list.clear();
    if (ctx->staged_pending) {
        CK(cudaEventSynchronize(ctx->staged));
        ctx->staged_pending = false;
    }
    // M1 models whose [Fe/H] falls between grid points get their own interpolated isochrones
    std::vector<int> m1_k(n_sets, -1);
    std::vector<double> m1_t(n_sets, 0.0);
    uint32_t n_m1 = 0;
    for (int s = 0; s < n_sets; ++s) {
        if (p[s].feh_sigma > 0.0) continue;
        double t;
        const int k = m.m1_bracket(p[s].feh_mean, t);
        if (t > 0.0) {
            m1_k[s] = k;
            m1_t[s] = t;
            ++n_m1;
        }
    }
    const size_t iso_pts = (size_t)m.n_ages * m.n_mass;
    const size_t in_bytes = sizeof(TabSetIn) * n_sets, w_bytes = sizeof(double) * (size_t)nw * n_sets;
    const size_t m1_bytes = sizeof(double) * iso_pts * (1 + B) * n_m1;
    const size_t desc_off = (in_bytes + w_bytes + m1_bytes + 255) & ~size_t(255);
    const size_t up_bytes = desc_off + sizeof(SetDesc) * n_sets;   // one upload: inputs + descriptors
    CK(ctx->h_tab_in.ensure(up_bytes));
    TabSetIn *tin = ctx->h_tab_in.as<TabSetIn>();
    double *wts = reinterpret_cast<double *>(ctx->h_tab_in.as<uint8_t>() + in_bytes);
    double *m1_imf = wts + (size_t)nw * n_sets, *m1_flux = m1_imf + iso_pts * n_m1;
    std::vector<double> mdf;
    uint64_t img_off = 0;
    uint32_t m1_i = 0;
    const bool pool = (ctx->cfg.flags & PCMD_FLAG_POOL) != 0;
    bool any_dense = false, any_ptrs = false;
    uint64_t btab_bytes = 0;      // word tables of every set's dense groups
    for (int s = 0; s < n_sets; ++s) {
        tin[s].m1_k = m1_k[s];
        tin[s].m1_off = 0;
        if (m1_k[s] >= 0) {
            tin[s].m1_off = (uint32_t)(m1_i * iso_pts);
            m.m1_isochrone(m1_k[s], m1_t[s], m1_imf + m1_i * iso_pts, m1_flux + m1_i * iso_pts * B);
            ++m1_i;
        }
        m.mdf_weights(p[s].feh_mean, p[s].feh_sigma, mdf);
        double *w = wts + (size_t)s * nw;
        for (int j = 0; j < m.n_ages; ++j) {
            const double sfh = std::pow(10.0, p[s].log_sfh[j]);
            for (int k = 0; k < m.n_feh; ++k) w[j * m.n_feh + k] = sfh * mdf[k];
        }
        uint32_t btab_cap = 0;
        {   // an upper bound of the largest lambda: can the model have dense inversion groups or
            // transformed-rejection points (the draw kernel's full instantiation), or only sparse
            // inversion groups?
            double bound = 0.0;
            for (int j = 0; j < m.n_ages; ++j)
                for (int k = 0; k < m.n_feh; ++k) {
                    double im = m.imf_max[(size_t)j * m.n_feh + k];
                    if (k == m1_k[s]) {
                        im = 0.0;
                        const double *mi = m1_imf + (size_t)tin[s].m1_off + (size_t)j * m.n_mass;
                        for (int i = 0; i < m.n_mass; ++i) im = std::max(im, mi[i]);
                    }
                    bound = std::max(bound, w[j * m.n_feh + k] * im);
                }
            const double top = bound * std::max(hf[0], hf[1]);
            if (top >= 0.999 * (double)kDenseLam) any_dense = true;
            if (top >= 0.999 * (double)kPtrsThreshold) any_ptrs = true;
            // room for the dense groups' word tables: a dense group holds a point whose lambda
            // bound reaches kDenseLam, so the count of such points (the sorted IMF weights of
            // each isochrone, binary search) bounds the dense list of either half
            uint64_t pts = 0;
            if (top >= 0.999 * (double)kDenseLam) {
                const double hmax = std::max(hf[0], hf[1]);
                for (int j = 0; j < m.n_ages; ++j)
                    for (int k = 0; k < m.n_feh; ++k) {
                        const double sw = w[j * m.n_feh + k] * hmax;
                        if (!(sw > 0.0)) continue;
                        const double cut = 0.999 * (double)kDenseLam / sw;
                        if (k == m1_k[s]) {
                            const double *mi = m1_imf + (size_t)tin[s].m1_off + (size_t)j * m.n_mass;
                            for (int i = 0; i < m.n_mass; ++i) pts += mi[i] >= cut ? 1u : 0u;
                        } else {
                            const double *dsc = m.imf_desc.data() + ((size_t)j * m.n_feh + k) * m.n_mass;
                            pts += (uint64_t)(std::upper_bound(dsc, dsc + m.n_mass, cut, std::greater<double>()) - dsc);
                        }
                    }
            }
            btab_cap = (uint32_t)std::min<uint64_t>(pts, (P + kGroup - 1u) / kGroup);
        }
        tin[s].base = (uint64_t)s * L.bytes;
        tin[s].flux_factor = std::pow(10.0, -0.4 * p[s].dmod);
        tin[s].w_off = (uint32_t)(s * nw);
        tin[s].pad = 0;
        SetDesc &d = ctx->descs[s];
        std::memset(&d, 0, sizeof d);
        for (int h = 0; h < 2; ++h) {
            d.grp_off[h] = tin[s].base + L.grp_off[h];
            d.dense_off[h] = tin[s].base + L.dense_off[h];
            d.slow_off[h] = tin[s].base + L.slow_off[h];
            d.ptrs_off[h] = tin[s].base + L.ptrs_off[h];
        }
        d.tail_off = tin[s].base + L.tail_off;
        d.flux_off = tin[s].base + L.flux_off;
        d.btab_cap = btab_cap;
        for (int h = 0; h < 2; ++h) d.btab_off[h] = btab_bytes + (uint64_t)h * btab_cap * kBtabGroupBytes;
        btab_bytes += 2ull * btab_cap * kBtabGroupBytes;
        d.pool_on = (ctx->cfg.flags & PCMD_FLAG_POOL) ? 1u : 0u;
        for (int h = 0; h < 2; ++h) d.pool_off[h] = tin[s].base + L.pool_off[h];
        // dust screen of this model (Section 2.2): E = 10^log_ebv exp(sigma z)
        d.dust_on = m.dust ? 1u : 0u;
        d.dust_a = (float)(std::log(10.0) * p[s].log_ebv);
        d.dust_sigma = (float)p[s].dust_sigma;
        for (int b = 0; b < kMaxBands; ++b) d.dust_c[b] = b < B ? (float)(-0.4 * m.r_ext[b]) : 0.0f;
        d.n_im = (uint32_t)n_im[s];
        d.set_id = first_set_id + (uint32_t)s;
        d.img_off = img_off;
        img_off += (uint64_t)B * n_im[s] * n_im[s];
        const uint32_t npix = (uint32_t)n_im[s] * (uint32_t)n_im[s];
        d.item_begin = (uint32_t)ctx->item_list.size();
        d.n_items = (npix + ppc - 1) / ppc;
        for (uint32_t t = 0; t < d.n_items; ++t) ctx->item_list.push_back(make_uint2((uint32_t)s, t));
        if (cost_sorted && n_sets > 1) ctx->cost[s] = model_cost(m, w, hf);
    }
    const size_t n_items = ctx->item_list.size();
    ctx->order_list.resize(n_items);
    std::iota(ctx->order_list.begin(), ctx->order_list.end(), 0u);
    if (cost_sorted && n_sets > 1) {
        std::stable_sort(ctx->order_list.begin(), ctx->order_list.end(), [&](uint32_t a, uint32_t b) {
            return ctx->cost[ctx->item_list[a].x] > ctx->cost[ctx->item_list[b].x];
        });
    }
    const uint32_t G = (P + kGroup - 1u) / kGroup;
    CK(ctx->h_items.ensure(sizeof(uint2) * n_items));
    CK(ctx->h_order.ensure(sizeof(uint32_t) * n_items));
    CK(ctx->tables.ensure(L.bytes * (size_t)n_sets));
    // the total-count sampler replaces the inversion groups (no dense groups to draw); points at or
    // above the rejection boundary keep their own draws either way
    const int draw_paths = pool ? (kPathPool | (any_ptrs ? kPathDense : 0)) : (any_dense ? kPathDense : kPathSparse);
    const bool need_btab = !pool && any_dense;
    if (need_btab) CK(ctx->btab.ensure((size_t)btab_bytes));
    CK(ctx->tab_in.ensure(up_bytes));
    ctx->desc_d = reinterpret_cast<SetDesc *>(ctx->tab_in.as<uint8_t>() + desc_off);
    const size_t n_scr = (ctx->cfg.flags & PCMD_FLAG_POOL) ? 2 : 1;
    const size_t grp_scr = 2 * (size_t)G * n_sets * n_scr, pt_scr = 2 * (size_t)G * kGroup * n_sets;
    CK(ctx->tab_scratch.ensure(sizeof(uint4) * (grp_scr + pt_scr)));
    CK(ctx->items.ensure(sizeof(uint2) * n_items));
    CK(ctx->order.ensure(sizeof(uint32_t) * n_items));
    std::memcpy(ctx->h_tab_in.as<uint8_t>() + desc_off, ctx->descs.data(), sizeof(SetDesc) * n_sets);
    std::memcpy(ctx->h_items.p, ctx->item_list.data(), sizeof(uint2) * n_items);
    std::memcpy(ctx->h_order.p, ctx->order_list.data(), sizeof(uint32_t) * n_items);
    CK(cudaMemcpyAsync(ctx->tab_in.p, ctx->h_tab_in.p, up_bytes, cudaMemcpyHostToDevice, ctx->st));
    CK(upload_if_changed(ctx->up_items, ctx->items, ctx->h_items.p, sizeof(uint2) * n_items, ctx->st));
    CK(upload_if_changed(ctx->up_order, ctx->order, ctx->h_order.p, sizeof(uint32_t) * n_items, ctx->st));
    CK(cudaEventRecord(ctx->staged, ctx->st));
    ctx->staged_pending = true;

    TabArgs ta;
    std::memset(&ta, 0, sizeof ta);
    ta.tables = ctx->tables.as<uint8_t>();
    ta.btab = need_btab ? ctx->btab.as<uint8_t>() : nullptr;
    ta.err = ctx->err.as<uint32_t>();
    ta.desc = ctx->desc_d;
    ta.sets = ctx->tab_in.as<TabSetIn>();
    ta.weights = reinterpret_cast<const double *>(ctx->tab_in.as<uint8_t>() + in_bytes);
    ta.imf = ctx->imf_d.as<double>();
    ta.base_flux = ctx->bflux_d.as<double>();
    ta.m1_imf = reinterpret_cast<const double *>(ctx->tab_in.as<uint8_t>() + in_bytes + w_bytes);
    ta.m1_flux = ta.m1_imf + iso_pts * n_m1;
    ta.hf[0] = hf[0];
    ta.hf[1] = hf[1];
    ta.P = P;
    ta.G = G;
    ta.n_mass = m.n_mass;
    ta.n_feh = m.n_feh;
    ta.n_bands = B;
    ta.layout = L;
    ta.scratch = ctx->tab_scratch.as<uint4>();
    ta.insp_lam = insp_lam;
    ta.insp_flux = insp_flux;
    ta.insp_z0 = insp_z0;
    ta.pool = (ctx->cfg.flags & PCMD_FLAG_POOL) ? 1 : 0;
    ta.pool_scratch = ta.pool ? ta.scratch + 2 * (size_t)G * n_sets : nullptr;
    ta.pt_scratch = ta.scratch + grp_scr;
    {
        KTimer t(ctx, PCMD_K_TABLES, ctx->st);
        CK(launch_build_tables(ta, n_sets, ctx->st));
        t.done(ctx->st);
    }
    ctx->n_sets = n_sets;
    ctx->draw_paths = draw_paths;
    ctx->n_im.assign(n_im, n_im + n_sets);
    return PCMD_OK;
}

static DrawArgs base_draw_args(pcmd_ctx *ctx) {
    DrawArgs a;
    std::memset(&a, 0, sizeof a);
    a.tables = ctx->tables.as<uint8_t>();
    a.btab = ctx->btab.as<uint8_t>();
    a.desc = ctx->desc_d;
    a.items = ctx->items.as<uint2>();
    a.order = ctx->order.as<uint32_t>();
    a.n_items = (uint32_t)ctx->item_list.size();
    a.queue = ctx->queue.as<uint32_t>();
    a.seed = ctx->cfg.seed;
    for (int r = 0; r < 10; ++r) {
        a.rk0[r] = (uint32_t)ctx->cfg.seed + (uint32_t)r * 0x9E3779B9u;
        a.rk1[r] = (uint32_t)(ctx->cfg.seed >> 32) + (uint32_t)r * 0xBB67AE85u;
    }
    a.err = ctx->err.as<uint32_t>();
    a.chunk = ctx->chunk;
    a.split = ctx->split;
    a.n_points = (uint32_t)ctx->model.n_points();
    a.ptrs_cap = ctx->ptrs_cap;
    a.pc = pixel_consts(ctx);
    return a;
}

static pcmd_status launch_draw_mode(pcmd_ctx *ctx, DrawArgs &a, int mode) {
    const int B = ctx->model.n_bands;
    const bool kahan = (ctx->cfg.flags & PCMD_FLAG_KAHAN) != 0;
    const size_t smem = draw_smem_bytes(B, ctx->chunk, ctx->block, ctx->split, mode, ctx->cfg.hess_nx,
                                        ctx->cfg.hess_ny);
    int per_sm = draw_max_blocks_per_sm(B, kahan, mode, ctx->draw_paths, ctx->block, smem);
    if (per_sm < 1) per_sm = 1;
    int grid = std::min<int>((int)a.n_items, per_sm * ctx->n_sm);
    if (grid < 1) grid = 1;
    CK(cudaMemsetAsync(ctx->queue.p, 0, sizeof(uint32_t), ctx->st));
    KTimer t(ctx, PCMD_K_DRAW, ctx->st);
    CK(launch_draw(a, B, kahan, mode, ctx->draw_paths, grid, ctx->block, smem, ctx->st));
    t.done(ctx->st);
    return PCMD_OK;
}

extern "C" {

pcmd_status pcmd_create(const pcmd_config *cfg, pcmd_ctx **out) {
    if (!out) return PCMD_ERR_ARG;
    *out = nullptr;
    if (!cfg) return PCMD_ERR_ARG;
    const pcmd_config &c = *cfg;
    if (c.n_bands < 2 || c.n_bands > PCMD_MAX_BANDS) return PCMD_ERR_ARG;
    if (c.n_ages < 1 || c.n_ages > PCMD_MAX_SFH || c.n_feh < 1 || c.n_mass < 1) return PCMD_ERR_ARG;
    if ((long long)c.n_ages * c.n_feh * c.n_mass > (1LL << 24)) return PCMD_ERR_ARG;
    if (!c.feh_grid || !c.mass || !c.abs_mag) return PCMD_ERR_ARG;
    if (!is_fin(c.imf_slope) || !is_fin(c.f_dust) || c.f_dust < 0.0 || c.f_dust > 1.0) return PCMD_ERR_ARG;
    if (c.imf != PCMD_IMF_POWER && c.imf != PCMD_IMF_KROUPA) return PCMD_ERR_ARG;
    if (!is_fin(c.mdf_cut) || c.mdf_cut < 0.0 || c.mdf_cut >= 1.0) return PCMD_ERR_ARG;
    if (c.hess_nx < 1 || c.hess_ny < 1 || (long long)c.hess_nx * c.hess_ny > 40000) return PCMD_ERR_ARG;
    if (!(c.hess_width > 0.0) || !is_fin(c.hess_width) || !is_fin(c.hess_c_lo) || !is_fin(c.hess_m_lo))
        return PCMD_ERR_ARG;
    if (c.max_im < 1 || c.max_im > 16384 || c.max_sets < 1 || c.max_sets > 65535) return PCMD_ERR_ARG;
    if (c.psf && (c.psf_size < 1 || c.psf_size > PCMD_MAX_PSF || (c.psf_size & 1) == 0)) return PCMD_ERR_ARG;
    if (c.psf_grid != 0 && c.psf_grid != 1 && c.psf_grid != 4) return PCMD_ERR_ARG;
    const size_t P = (size_t)c.n_ages * c.n_feh * c.n_mass;
    for (int b = 0; b < c.n_bands; ++b)
        if (!(c.exptime[b] > 0.0) || !is_fin(c.exptime[b]) || !is_fin(c.zeropoint[b]) ||
            !is_fin(c.sky[b]) || c.sky[b] < 0.0 ||
            !is_fin(c.r_ext[b]))
            return PCMD_ERR_ARG;
    for (size_t i = 0; i < P; ++i) {
        if (!(c.mass[i] > 0.0) || !is_fin(c.mass[i])) return PCMD_ERR_ARG;
        if (i % c.n_mass && !(c.mass[i] > c.mass[i - 1])) return PCMD_ERR_ARG;
        for (int b = 0; b < c.n_bands; ++b)
            if (!is_fin(c.abs_mag[i * c.n_bands + b])) return PCMD_ERR_ARG;
    }
    for (int k = 0; k < c.n_feh; ++k)
        if (!is_fin(c.feh_grid[k]) || (k > 0 && !(c.feh_grid[k] > c.feh_grid[k - 1]))) return PCMD_ERR_ARG;

    pcmd_ctx *ctx = new pcmd_ctx();
    ctx->cfg = c;
    Model &m = ctx->model;
    m.n_bands = c.n_bands;
    m.n_ages = c.n_ages;
    m.n_feh = c.n_feh;
    m.n_mass = c.n_mass;
    m.feh.assign(c.feh_grid, c.feh_grid + c.n_feh);
    m.mass.assign(c.mass, c.mass + P);
    m.abs_mag.assign(c.abs_mag, c.abs_mag + P * c.n_bands);
    m.imf_slope = c.imf_slope;
    m.imf_kind = c.imf;
    m.mdf_cut = c.mdf_cut;
    m.f_dust = c.f_dust;
    m.dust = (c.flags & PCMD_FLAG_DUST) != 0;
    for (int b = 0; b < kMaxBands; ++b) {
        m.exptime[b] = b < c.n_bands ? c.exptime[b] : 1.0;
        m.zeropoint[b] = b < c.n_bands ? c.zeropoint[b] : 0.0;
        m.r_ext[b] = b < c.n_bands ? c.r_ext[b] : 0.0;
    }
    m.build_imf();
    m.build_base_flux();
    ctx->cfg.feh_grid = nullptr;
    ctx->cfg.mass = nullptr;
    ctx->cfg.abs_mag = nullptr;
    ctx->cfg.log_age = nullptr;
    ctx->cfg.psf = nullptr;
    if (c.psf) {
        const size_t n_kern = c.psf_grid == 4 ? 16 : 1;
        ctx->psf.assign(c.psf, c.psf + n_kern * c.n_bands * c.psf_size * c.psf_size);
        if (c.psf_size == 25 && n_kern == 1) {
            ctx->psf25.assign((size_t)kMaxBands * 625, 0.0f);
            std::copy(ctx->psf.begin(), ctx->psf.end(), ctx->psf25.begin());
        }
    }
    ctx->st = (cudaStream_t)c.stream;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
        delete ctx;
        return PCMD_ERR_CUDA;
    }
    float st16[16];
    stirlerr_table(st16);
    pcmd_status rc = PCMD_OK;
    do {
        if (upload_stirlerr(st16) != cudaSuccess) { rc = PCMD_ERR_CUDA; break; }
        if (cudaEventCreateWithFlags(&ctx->staged, cudaEventDisableTiming) != cudaSuccess) { rc = PCMD_ERR_CUDA; break; }
        if (cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking) != cudaSuccess) { rc = PCMD_ERR_CUDA; break; }
        if (ctx->err.ensure(sizeof(uint32_t)) != cudaSuccess || ctx->queue.ensure(sizeof(uint32_t)) != cudaSuccess) { rc = PCMD_ERR_OOM; break; }
        if (cudaMemset(ctx->err.p, 0, sizeof(uint32_t)) != cudaSuccess) { rc = PCMD_ERR_CUDA; break; }
        if (!ctx->psf.empty()) {
            if (ctx->psf_d.ensure(ctx->psf.size() * 4) != cudaSuccess) { rc = PCMD_ERR_OOM; break; }
            if (cudaMemcpy(ctx->psf_d.p, ctx->psf.data(), ctx->psf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) { rc = PCMD_ERR_CUDA; break; }
        }
        if (ctx->h_ll.ensure(sizeof(double) * c.max_sets + 16) != cudaSuccess) { rc = PCMD_ERR_OOM; break; }
        if (ctx->imf_d.ensure(sizeof(double) * P) != cudaSuccess ||
            ctx->bflux_d.ensure(sizeof(double) * P * c.n_bands) != cudaSuccess) { rc = PCMD_ERR_OOM; break; }
        if (cudaMemcpy(ctx->imf_d.p, m.imf.data(), sizeof(double) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ctx->bflux_d.p, m.base_flux.data(), sizeof(double) * P * c.n_bands,
                       cudaMemcpyHostToDevice) != cudaSuccess) { rc = PCMD_ERR_CUDA; break; }
        ctx->layout = tab_layout((uint32_t)P, c.n_bands);
        if (ctx->h_meta.ensure(sizeof(uint64_t) * (size_t)c.max_sets * 3) != cudaSuccess) { rc = PCMD_ERR_OOM; break; }
    } while (0);
    if (rc != PCMD_OK) {
        pcmd_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return PCMD_OK;
}

void pcmd_destroy(pcmd_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->st);
    for (auto &g : ctx->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (int k = 0; k < PCMD_KERNEL_KINDS; ++k)
        for (auto &pr : ctx->ev[k]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    DevBuf *bufs[] = {&ctx->ll_part, &ctx->ll_ticket, &ctx->tables, &ctx->btab, &ctx->items, &ctx->order, &ctx->partials,
                      &ctx->part_begin, &ctx->part_count, &ctx->image, &ctx->pix_off, &ctx->hess,
                      &ctx->moments, &ctx->counters, &ctx->ll, &ctx->psf_d, &ctx->queue, &ctx->err,
                      &ctx->imf_d, &ctx->bflux_d, &ctx->tab_in, &ctx->tab_scratch, &ctx->insp};
    for (DevBuf *b : bufs) b->release();
    HostBuf *hb[] = {&ctx->h_tab_in, &ctx->h_items, &ctx->h_order, &ctx->h_meta, &ctx->h_ll};
    for (HostBuf *b : hb) b->release();
    if (ctx->staged) cudaEventDestroy(ctx->staged);
    if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
    delete ctx;
}

const char *pcmd_last_error(const pcmd_ctx *ctx) { return ctx ? ctx->err_text.c_str() : "no context"; }

int pcmd_n_points(const pcmd_ctx *ctx) { return ctx ? ctx->model.n_points() : 0; }

pcmd_status pcmd_profile(pcmd_ctx *ctx, int enable) {
    if (!ctx) return PCMD_ERR_ARG;
    ctx->profiling = enable != 0;
    return PCMD_OK;
}

pcmd_status pcmd_kernel_times(pcmd_ctx *ctx, double *h_ms, int *h_count) {
    if (!ctx || !h_ms || !h_count) return PCMD_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st));
    for (int k = 0; k < PCMD_KERNEL_KINDS; ++k) {
        double ms = 0.0;
        for (auto &pr : ctx->ev[k]) {
            float v = 0.0f;
            if (cudaEventElapsedTime(&v, pr.first, pr.second) == cudaSuccess) ms += v;
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        h_ms[k] = ms;
        h_count[k] = (int)ctx->ev[k].size();
        ctx->ev[k].clear();
    }
    return PCMD_OK;
}

pcmd_status pcmd_set_launch(pcmd_ctx *ctx, int block, int split, int chunk) {
    if (!ctx) return PCMD_ERR_ARG;
    if (block < 32 || block > 256 || block % 32) return arg_error(ctx, "block must be 32..256, a multiple of 32");
    if (split < 1 || block % (split * 32)) return arg_error(ctx, "block / split must be a multiple of 32");
    if (chunk < 1 || chunk > 256) return arg_error(ctx, "chunk must be 1..256");
    ctx->block = block;
    ctx->split = split;
    ctx->chunk = chunk;
    return PCMD_OK;
}

pcmd_status pcmd_set_attempt_cap(pcmd_ctx *ctx, int cap) {
    if (!ctx) return PCMD_ERR_ARG;
    if (cap < 0 || cap > (int)kPtrsMaxAttempts) return arg_error(ctx, "attempt cap must be 0..1024");
    ctx->ptrs_cap = cap == 0 ? kPtrsMaxAttempts : (uint32_t)cap;
    return PCMD_OK;
}

pcmd_status pcmd_simulate(pcmd_ctx *ctx, const pcmd_params *h_params, int n_sets, const int *h_n_im,
                          uint32_t first_set_id, float *d_image) {
    if (!ctx) return PCMD_ERR_ARG;
    pcmd_status rc = check_params(ctx, h_params, n_sets, h_n_im);
    if (rc != PCMD_OK) return rc;
    const int ppc = ctx->block / ctx->split;
    rc = stage_sets(ctx, h_params, n_sets, h_n_im, first_set_id, n_sets > 1, ppc);
    if (rc != PCMD_OK) return rc;
    size_t floats = 0;
    for (int s = 0; s < n_sets; ++s) floats += (size_t)ctx->model.n_bands * h_n_im[s] * h_n_im[s];
    float *img = d_image;
    if (!img) {
        CK(ctx->image.ensure(floats * 4));
        img = ctx->image.as<float>();
    }
    DrawArgs a = base_draw_args(ctx);
    a.image = img;
    rc = launch_draw_mode(ctx, a, kModeImage);
    if (rc != PCMD_OK) return rc;
    ctx->img_ptr = img;
    ctx->have_images = true;
    ctx->have_hess = false;
    return PCMD_OK;
}

pcmd_status pcmd_hess(pcmd_ctx *ctx, uint32_t *d_hess, double *d_moments, uint32_t *d_counters,
                      float *d_pixels) {
    if (!ctx) return PCMD_ERR_ARG;
    if (!ctx->have_images) {
        ctx->err_text = "pcmd_hess needs a preceding pcmd_simulate";
        return PCMD_ERR_STATE;
    }
    const int n_sets = ctx->n_sets;
    const int nbins = ctx->cfg.hess_nx * ctx->cfg.hess_ny;
    if (!d_hess) CK(ctx->hess.ensure(sizeof(uint32_t) * nbins * n_sets));
    if (!d_moments) CK(ctx->moments.ensure(sizeof(double) * 3 * n_sets));
    if (!d_counters) CK(ctx->counters.ensure(sizeof(uint32_t) * 2 * n_sets));
    uint32_t *hh = d_hess ? d_hess : ctx->hess.as<uint32_t>();
    double *mm = d_moments ? d_moments : ctx->moments.as<double>();
    uint32_t *cc = d_counters ? d_counters : ctx->counters.as<uint32_t>();
    int max_tiles = 1;
    for (int s = 0; s < n_sets; ++s) max_tiles = std::max(max_tiles, hess_tiles(ctx->n_im[s]));
    int cps = std::max(1, (2 * ctx->n_sm + n_sets - 1) / n_sets);
    cps = std::min(cps, max_tiles);
    // per-set partial ranges and pixel-output offsets (pinned host staging, then device)
    if (ctx->staged_pending) {
        CK(cudaEventSynchronize(ctx->staged));
        ctx->staged_pending = false;
    }
    CK(ctx->h_meta.ensure(sizeof(uint64_t) * (size_t)n_sets * 3));
    uint32_t *hb = ctx->h_meta.as<uint32_t>();
    uint32_t *hc = hb + n_sets;
    uint64_t *hp = reinterpret_cast<uint64_t *>(ctx->h_meta.as<uint8_t>() + ((sizeof(uint32_t) * 2 * n_sets + 7) & ~size_t(7)));
    uint64_t po = 0;
    for (int s = 0; s < n_sets; ++s) {
        hb[s] = (uint32_t)(s * cps);
        hc[s] = (uint32_t)cps;
        hp[s] = po;
        po += (uint64_t)(ctx->model.n_bands + 2) * ctx->n_im[s] * ctx->n_im[s];
    }
    CK(ctx->part_begin.ensure(sizeof(uint32_t) * n_sets));
    CK(ctx->part_count.ensure(sizeof(uint32_t) * n_sets));
    CK(ctx->pix_off.ensure(sizeof(uint64_t) * n_sets));
    CK(ctx->partials.ensure(sizeof(double) * 3 * (size_t)cps * n_sets));
    CK(upload_if_changed(ctx->up_part_begin, ctx->part_begin, hb, sizeof(uint32_t) * n_sets, ctx->st));
    CK(upload_if_changed(ctx->up_part_count, ctx->part_count, hc, sizeof(uint32_t) * n_sets, ctx->st));
    CK(upload_if_changed(ctx->up_pix_off, ctx->pix_off, hp, sizeof(uint64_t) * n_sets, ctx->st));
    CK(cudaEventRecord(ctx->staged, ctx->st));
    ctx->staged_pending = true;
    CK(cudaMemsetAsync(hh, 0, sizeof(uint32_t) * nbins * n_sets, ctx->st));
    CK(cudaMemsetAsync(cc, 0, sizeof(uint32_t) * 2 * n_sets, ctx->st));
    HessArgs h;
    std::memset(&h, 0, sizeof h);
    h.image = ctx->img_ptr;
    h.desc = ctx->desc_d;
    h.n_sets = n_sets;
    h.n_bands = ctx->model.n_bands;
    h.psf = ctx->psf.empty() ? nullptr : ctx->psf_d.as<float>();
    h.psf_size = ctx->psf.empty() ? 0 : ctx->cfg.psf_size;
    h.psf_grid = ctx->cfg.psf_grid == 4 ? 4 : 1;
    h.hess = hh;
    h.counters = cc;
    h.cta_moments = ctx->partials.as<double>();
    h.ctas_per_set = cps;
    h.pixels = d_pixels;
    h.pix_off = ctx->pix_off.as<uint64_t>();
    h.pc = pixel_consts(ctx);
    {
        KTimer t(ctx, PCMD_K_HESS, ctx->st);
        CK(launch_hess(h, ctx->psf25.empty() ? nullptr : ctx->psf25.data(), ctx->st));
        t.done(ctx->st);
    }
    {
        KTimer t(ctx, PCMD_K_FINALIZE, ctx->st);
        CK(launch_moments_finalize(ctx->partials.as<double>(), ctx->part_begin.as<uint32_t>(),
                                   ctx->part_count.as<uint32_t>(), n_sets, mm, ctx->st));
        t.done(ctx->st);
    }
    ctx->hess_ptr = hh;
    ctx->mom_ptr = mm;
    ctx->ctr_ptr = cc;
    ctx->have_hess = true;
    return PCMD_OK;
}

pcmd_status pcmd_sync(pcmd_ctx *ctx) {
    if (!ctx) return PCMD_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st));
    uint32_t e = 0;
    CK(cudaMemcpy(&e, ctx->err.p, sizeof e, cudaMemcpyDeviceToHost));
    if (e) {
        CK(cudaMemset(ctx->err.p, 0, sizeof(uint32_t)));
        if (e & kErrTimeout) {
            ctx->err_text = "a bounded wait inside a kernel ran out";
            return PCMD_ERR_TIMEOUT;
        }
        if (e & kErrBounds) {
            ctx->err_text = "a dense-group list exceeded the room reserved for its word tables";
            return PCMD_ERR_CUDA;
        }
        ctx->err_text = "transformed rejection reached its attempt cap";
        return PCMD_ERR_SAMPLER_LIMIT;
    }
    return PCMD_OK;
}

// Partials and tickets of the likelihood launch; tickets are zeroed when (re)allocated and
// left at zero by every launch.
static pcmd_status ensure_ll_scratch(pcmd_ctx *ctx, int n_sets) {
    const int nbins = ctx->cfg.hess_nx * ctx->cfg.hess_ny;
    const int ctas = loglike_ctas_per_set(n_sets, nbins);
    CK(ctx->ll_part.ensure(sizeof(double) * (size_t)ctas * n_sets));
    const uint64_t gen = ctx->ll_ticket.gen;
    CK(ctx->ll_ticket.ensure(sizeof(uint32_t) * (size_t)n_sets));
    if (ctx->ll_ticket.gen != gen) CK(cudaMemsetAsync(ctx->ll_ticket.p, 0, ctx->ll_ticket.cap, ctx->st));
    return PCMD_OK;
}

// Likelihoods and the kernels' error word back to pinned host memory in one stream round trip.
static pcmd_status fetch_ll(pcmd_ctx *ctx, int n_sets, double *h_ll) {
    double *hl = ctx->h_ll.as<double>();
    uint32_t *he = reinterpret_cast<uint32_t *>(hl + n_sets);
    CK(cudaMemcpyAsync(hl, ctx->ll.p, sizeof(double) * n_sets, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(he, ctx->err.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const uint32_t e = *he;
    std::memcpy(h_ll, hl, sizeof(double) * n_sets);
    if (!e) return PCMD_OK;
    CK(cudaMemset(ctx->err.p, 0, sizeof(uint32_t)));
    if (e & kErrTimeout) {
        ctx->err_text = "a bounded wait inside a kernel ran out";
        return PCMD_ERR_TIMEOUT;
    }
    if (e & kErrBounds) {
        ctx->err_text = "a dense-group list exceeded the room reserved for its word tables";
        return PCMD_ERR_CUDA;
    }
    ctx->err_text = "transformed rejection reached its attempt cap";
    return PCMD_ERR_SAMPLER_LIMIT;
}

static pcmd_status check_mock(pcmd_ctx *ctx, const uint32_t *d_mock, const double *mom, double npix,
                              int mode, double *h_ll) {
    if (!d_mock || !mom || !h_ll) return arg_error(ctx, "mock Hess, mock moments and h_ll are required");
    if (!(npix > 0.0) || !is_fin(npix)) return arg_error(ctx, "mock_n_pix must be positive");
    if (mode != PCMD_LL_PAPER && mode != PCMD_LL_POISSON) return arg_error(ctx, "unknown likelihood mode");
    return PCMD_OK;
}

pcmd_status pcmd_loglike(pcmd_ctx *ctx, const uint32_t *d_mock_hess, const double *h_mock_moments,
                         double mock_n_pix, int mode, double *h_ll) {
    if (!ctx) return PCMD_ERR_ARG;
    pcmd_status rc = check_mock(ctx, d_mock_hess, h_mock_moments, mock_n_pix, mode, h_ll);
    if (rc != PCMD_OK) return rc;
    if (!ctx->have_hess) {
        ctx->err_text = "pcmd_loglike needs a preceding pcmd_hess";
        return PCMD_ERR_STATE;
    }
    const int n_sets = ctx->n_sets;
    CK(ctx->ll.ensure(sizeof(double) * n_sets));
    rc = ensure_ll_scratch(ctx, n_sets);
    if (rc != PCMD_OK) return rc;
    {
        KTimer t(ctx, PCMD_K_LOGLIKE, ctx->st);
        CK(launch_loglike(ctx->hess_ptr, ctx->mom_ptr, ctx->desc_d, n_sets,
                          ctx->cfg.hess_nx * ctx->cfg.hess_ny, d_mock_hess, h_mock_moments[0],
                          h_mock_moments[1], h_mock_moments[2], mock_n_pix, mode,
                          (ctx->cfg.flags & PCMD_FLAG_SIGMA_SQRTSUM) ? 1 : 0, ctx->ll_part.as<double>(),
                          ctx->ll_ticket.as<uint32_t>(), ctx->ll.as<double>(), ctx->st));
        t.done(ctx->st);
    }
    return fetch_ll(ctx, n_sets, h_ll);
}

// Fused evaluation without a PSF: one persistent draw launch does draws, dust, noise,
// magnitudes and histograms of all sets; then moments and likelihoods.  The device-side
// sequence is captured once per shape into a CUDA graph and replayed.
static pcmd_status evaluate_fused(pcmd_ctx *ctx, int n_sets, const uint32_t *d_mock,
                                  const double *mom, double npix, int mode) {
    const int nbins = ctx->cfg.hess_nx * ctx->cfg.hess_ny;
    const size_t n_items = ctx->item_list.size();
    CK(ctx->hess.ensure(sizeof(uint32_t) * nbins * n_sets));
    CK(ctx->moments.ensure(sizeof(double) * 3 * n_sets));
    CK(ctx->counters.ensure(sizeof(uint32_t) * 2 * n_sets));
    CK(ctx->partials.ensure(sizeof(double) * 3 * n_items));
    CK(ctx->part_begin.ensure(sizeof(uint32_t) * n_sets));
    CK(ctx->part_count.ensure(sizeof(uint32_t) * n_sets));
    CK(ctx->ll.ensure(sizeof(double) * n_sets));
    const pcmd_status lrc = ensure_ll_scratch(ctx, n_sets);
    if (lrc != PCMD_OK) return lrc;
    CK(ctx->h_meta.ensure(sizeof(uint32_t) * 2 * n_sets + 16));
    uint32_t *hb = ctx->h_meta.as<uint32_t>();
    for (int s = 0; s < n_sets; ++s) {
        hb[s] = ctx->descs[s].item_begin;
        hb[n_sets + s] = ctx->descs[s].n_items;
    }
    CK(upload_if_changed(ctx->up_part_begin, ctx->part_begin, hb, sizeof(uint32_t) * n_sets, ctx->st));
    CK(upload_if_changed(ctx->up_part_count, ctx->part_count, hb + n_sets, sizeof(uint32_t) * n_sets, ctx->st));
    CK(cudaEventRecord(ctx->staged, ctx->st));
    ctx->staged_pending = true;

    const int B = ctx->model.n_bands;
    const bool kahan = (ctx->cfg.flags & PCMD_FLAG_KAHAN) != 0;
    const size_t smem = draw_smem_bytes(B, ctx->chunk, ctx->block, ctx->split, kModeFused,
                                        ctx->cfg.hess_nx, ctx->cfg.hess_ny);
    int per_sm = std::max(1, draw_max_blocks_per_sm(B, kahan, kModeFused, ctx->draw_paths, ctx->block, smem));
    const int grid = std::max(1, std::min<int>((int)n_items, per_sm * ctx->n_sm));
    uint64_t mk[4];
    std::memcpy(&mk[0], &mom[0], 8);
    std::memcpy(&mk[1], &mom[1], 8);
    std::memcpy(&mk[2], &mom[2], 8);
    std::memcpy(&mk[3], &npix, 8);
    const std::vector<size_t> key = {
        (size_t)n_sets, n_items, (size_t)grid, (size_t)mode, (size_t)ctx->block, (size_t)ctx->split,
        (size_t)ctx->chunk, (size_t)ctx->ptrs_cap, (size_t)ctx->draw_paths, mk[0], mk[1], mk[2], mk[3], (size_t)d_mock, (size_t)ctx->tables.p, (size_t)ctx->btab.p,
        (size_t)ctx->desc_d, (size_t)ctx->items.p, (size_t)ctx->order.p, (size_t)ctx->queue.p,
        (size_t)ctx->err.p, (size_t)ctx->hess.p, (size_t)ctx->counters.p, (size_t)ctx->partials.p,
        (size_t)ctx->part_begin.p, (size_t)ctx->part_count.p, (size_t)ctx->moments.p, (size_t)ctx->ll.p,
        (size_t)ctx->ll_part.p, (size_t)ctx->ll_ticket.p};
    cudaGraphExec_t gexec = nullptr;
    for (auto &g : ctx->graphs)
        if (g.key == key) {
            gexec = g.exec;
            g.used = ++ctx->graph_tick;
            break;
        }
    if (!gexec) {
        DrawArgs a = base_draw_args(ctx);
        a.hess = ctx->hess.as<uint32_t>();
        a.counters = ctx->counters.as<uint32_t>();
        a.item_moments = ctx->partials.as<double>();
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(ctx->cap_st, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(ctx->hess.p, 0, sizeof(uint32_t) * nbins * n_sets, ctx->cap_st);
        cudaMemsetAsync(ctx->counters.p, 0, sizeof(uint32_t) * 2 * n_sets, ctx->cap_st);
        cudaMemsetAsync(ctx->queue.p, 0, sizeof(uint32_t), ctx->cap_st);
        launch_draw(a, B, kahan, kModeFused, ctx->draw_paths, grid, ctx->block, smem, ctx->cap_st);
        launch_moments_finalize(ctx->partials.as<double>(), ctx->part_begin.as<uint32_t>(),
                                ctx->part_count.as<uint32_t>(), n_sets, ctx->moments.as<double>(),
                                ctx->cap_st);
        launch_loglike(ctx->hess.as<uint32_t>(), ctx->moments.as<double>(), ctx->desc_d,
                       n_sets, nbins, d_mock, mom[0], mom[1], mom[2], npix, mode,
                       (ctx->cfg.flags & PCMD_FLAG_SIGMA_SQRTSUM) ? 1 : 0, ctx->ll_part.as<double>(),
                       ctx->ll_ticket.as<uint32_t>(), ctx->ll.as<double>(), ctx->cap_st);
        CK(cudaStreamEndCapture(ctx->cap_st, &g));
        cudaError_t ec = cudaGraphInstantiate(&gexec, g, 0);
        cudaGraphDestroy(g);
        CK(ec);
        constexpr size_t kMaxGraphs = 32;
        if (ctx->graphs.size() >= kMaxGraphs) {
            size_t lru = 0;
            for (size_t i = 1; i < ctx->graphs.size(); ++i)
                if (ctx->graphs[i].used < ctx->graphs[lru].used) lru = i;
            cudaGraphExecDestroy(ctx->graphs[lru].exec);
            ctx->graphs.erase(ctx->graphs.begin() + (long)lru);
        }
        pcmd_ctx::GraphEntry ge;
        ge.key = key;
        ge.exec = gexec;
        ge.used = ++ctx->graph_tick;
        ctx->graphs.push_back(std::move(ge));
    }
    {
        KTimer t(ctx, PCMD_K_GRAPH, ctx->st);
        CK(cudaGraphLaunch(gexec, ctx->st));
        t.done(ctx->st);
    }
    ctx->hess_ptr = ctx->hess.as<uint32_t>();
    ctx->mom_ptr = ctx->moments.as<double>();
    ctx->ctr_ptr = ctx->counters.as<uint32_t>();
    ctx->have_hess = true;
    ctx->have_images = false;
    return PCMD_OK;
}

pcmd_status pcmd_evaluate(pcmd_ctx *ctx, const pcmd_params *h_params, int n_sets, const int *h_n_im,
                          uint32_t first_set_id, const uint32_t *d_mock_hess,
                          const double *h_mock_moments, double mock_n_pix, int mode, double *h_ll) {
    if (!ctx) return PCMD_ERR_ARG;
    pcmd_status rc = check_params(ctx, h_params, n_sets, h_n_im);
    if (rc != PCMD_OK) return rc;
    rc = check_mock(ctx, d_mock_hess, h_mock_moments, mock_n_pix, mode, h_ll);
    if (rc != PCMD_OK) return rc;
    if (!ctx->psf.empty()) {
        rc = pcmd_simulate(ctx, h_params, n_sets, h_n_im, first_set_id, nullptr);
        if (rc == PCMD_OK) rc = pcmd_hess(ctx, nullptr, nullptr, nullptr, nullptr);
        if (rc == PCMD_OK) rc = pcmd_loglike(ctx, d_mock_hess, h_mock_moments, mock_n_pix, mode, h_ll);
        return rc;
    }
    const int ppc = ctx->block / ctx->split;
    rc = stage_sets(ctx, h_params, n_sets, h_n_im, first_set_id, true, ppc);
    if (rc != PCMD_OK) return rc;
    rc = evaluate_fused(ctx, n_sets, d_mock_hess, h_mock_moments, mock_n_pix, mode);
    if (rc != PCMD_OK) return rc;
    return fetch_ll(ctx, n_sets, h_ll);
}

pcmd_status pcmd_sfh_bins(int model, const double *theta, int n_theta, int n_bins, const double *log_age_edges,
                          double *h_log_sfh) {
    return sfh_bins(model, theta, n_theta, n_bins, log_age_edges, h_log_sfh) ? PCMD_OK : PCMD_ERR_ARG;
}

pcmd_status pcmd_get_tables(pcmd_ctx *ctx, const pcmd_params *h_params, float *h_lam, float *h_flux,
                            uint32_t *h_z0) {
    if (!ctx || !h_params) return PCMD_ERR_ARG;
    int one = 1;
    pcmd_status rc = check_params(ctx, h_params, 1, &one);
    if (rc != PCMD_OK) return rc;
    // the device builder's own values (copies written while it builds the model's table)
    const size_t P = (size_t)ctx->model.n_points();
    const int B = ctx->model.n_bands;
    const size_t bytes = P * (2 * 4 + (size_t)B * 4 + 2 * 4);
    CK(ctx->insp.ensure(bytes));
    float *lam = ctx->insp.as<float>();
    float *flux = lam + 2 * P;
    uint32_t *z0 = reinterpret_cast<uint32_t *>(flux + P * B);
    rc = stage_sets(ctx, h_params, 1, &one, 0u, false, ctx->block / ctx->split, lam, flux, z0);
    if (rc != PCMD_OK) return rc;
    if (h_lam) CK(cudaMemcpyAsync(h_lam, lam, 2 * P * 4, cudaMemcpyDeviceToHost, ctx->st));
    if (h_flux) CK(cudaMemcpyAsync(h_flux, flux, P * B * 4, cudaMemcpyDeviceToHost, ctx->st));
    if (h_z0) CK(cudaMemcpyAsync(h_z0, z0, 2 * P * 4, cudaMemcpyDeviceToHost, ctx->st));
    return pcmd_sync(ctx);
}

pcmd_status pcmd_counts(pcmd_ctx *ctx, const pcmd_params *h_params, int n_im, uint32_t set_id,
                        uint32_t pix_begin, uint32_t n_pix, uint32_t *d_counts) {
    if (!ctx || !d_counts) return PCMD_ERR_ARG;
    pcmd_status rc = check_params(ctx, h_params, 1, &n_im);
    if (rc != PCMD_OK) return rc;
    const uint64_t npix = (uint64_t)n_im * n_im;
    if (n_pix == 0 || pix_begin >= npix || pix_begin + (uint64_t)n_pix > npix)
        return arg_error(ctx, "pixel range outside the image");
    const int ppc = ctx->block / ctx->split;
    rc = stage_sets(ctx, h_params, 1, &n_im, set_id, false, ppc);
    if (rc != PCMD_OK) return rc;
    // only the tiles that intersect the requested range
    const uint32_t t0 = pix_begin / ppc, t1 = (pix_begin + n_pix - 1) / ppc;
    std::vector<uint2> sub;
    for (uint32_t t = t0; t <= t1; ++t) sub.push_back(make_uint2(0u, t));
    CK(cudaEventSynchronize(ctx->staged));
    ctx->staged_pending = false;
    std::memcpy(ctx->h_items.p, sub.data(), sizeof(uint2) * sub.size());
    for (size_t i = 0; i < sub.size(); ++i) ctx->h_order.as<uint32_t>()[i] = (uint32_t)i;
    CK(upload_if_changed(ctx->up_items, ctx->items, ctx->h_items.p, sizeof(uint2) * sub.size(), ctx->st));
    CK(upload_if_changed(ctx->up_order, ctx->order, ctx->h_order.p, sizeof(uint32_t) * sub.size(), ctx->st));
    CK(cudaEventRecord(ctx->staged, ctx->st));
    ctx->staged_pending = true;
    const size_t P = (size_t)ctx->model.n_points();
    CK(cudaMemsetAsync(d_counts, 0, sizeof(uint32_t) * (size_t)n_pix * 2 * P, ctx->st));
    DrawArgs a = base_draw_args(ctx);
    a.n_items = (uint32_t)sub.size();
    a.counts = d_counts;
    a.count_pix0 = pix_begin;
    a.count_npix = n_pix;
    CK(ctx->image.ensure(sizeof(float) * ctx->model.n_bands * npix));
    a.image = ctx->image.as<float>();
    rc = launch_draw_mode(ctx, a, kModeCounts);
    ctx->have_images = false;
    ctx->have_hess = false;
    return rc;
}

pcmd_status pcmd_bin_mags(pcmd_ctx *ctx, const float *d_mag, const float *d_colour,
                          const uint8_t *d_valid, uint32_t n, uint32_t *d_hess, uint32_t *d_counters,
                          double *d_moments) {
    if (!ctx || !d_mag || !d_colour || !d_valid || !d_hess) return PCMD_ERR_ARG;
    const int nbins = ctx->cfg.hess_nx * ctx->cfg.hess_ny;
    CK(cudaMemsetAsync(d_hess, 0, sizeof(uint32_t) * nbins, ctx->st));
    if (d_counters) CK(cudaMemsetAsync(d_counters, 0, sizeof(uint32_t) * 2, ctx->st));
    if (d_moments) CK(cudaMemsetAsync(d_moments, 0, sizeof(double) * 3, ctx->st));
    if (n == 0) return PCMD_OK;
    const PixelConsts pc = pixel_consts(ctx);
    CK(launch_bin_mags(d_mag, d_colour, d_valid, n, d_hess, d_counters, d_moments, pc,
                       ctx->err.as<uint32_t>(), ctx->st));
    return PCMD_OK;
}

}  // extern "C"
