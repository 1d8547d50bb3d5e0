// Device table builder: the per-point part of the tables of every model of a call, built on the
// GPU from the host's per-isochrone weights (Section 2.1 / 2.2: lambda_jki = SFH_j MDF_k IMF_jk,i,
// split into the two dust halves) and the per-context FP64 IMF weights and base fluxes.
//
// Every FP64 step is one IEEE operation in the order of the host definition (explicit _rn
// intrinsics, nothing fused), so lambda, the fluxes and the thresholds equal the host's:
//   lambda_h,i = (float)((w_jk * imf_i) * hf_h),  flux_i,b = (float)(base_flux_i,b * 10^(-0.4 dmod))
//   p_0 = exp(-lambda), p_k = (p_{k-1} lambda) / k, F_k = F_{k-1} + p_k,
//   Z_k = ceil(F_k 2^32 - 1/2) - 1 (saturating at 2^32 - 1): n > k iff x > Z_k.
// Three launches: count (per point, reduced per 16-point group), scan (per model and half, the
// list positions of every group), write (group records, slow records, tail thresholds,
// transformed-rejection records at their positions).  One thread per point; the 16 points of
// a group are 16 consecutive lanes.
#include "common.cuh"
#include "tables_dev.h"

namespace pcmd {

namespace {

__device__ __forceinline__ uint32_t threshold_dev(double F) {
    const double y = __dsub_rn(__dmul_rn(F, 4294967296.0), 0.5);
    if (y >= 4294967295.0) return 0xFFFFFFFFu;
    const uint64_t t = (uint64_t)y;
    const uint64_t T = t + (y > (double)t ? 1u : 0u);
    return (uint32_t)(T - 1u);
}

struct PointIn {
    float lam;
    uint32_t i;
    bool valid;
};

__device__ __forceinline__ PointIn point_of(const TabArgs &a, const TabSetIn &in, uint32_t g, int j, int h) {
    PointIn p;
    p.i = g * (uint32_t)kGroup + (uint32_t)j;
    p.valid = p.i < a.P;
    p.lam = 0.0f;
    if (p.valid) {
        const double w = a.weights[in.w_off + p.i / (uint32_t)a.n_mass];
        const double lam = __dmul_rn(w, a.imf[p.i]);
        p.lam = (float)__dmul_rn(lam, a.hf[h]);
    }
    return p;
}

// Thresholds of an inversion point: calls f(k, Z_k) for k = 0 .. while Z_k < 2^32 - 1 (and the
// first saturated one), at most kInvCap values; returns Z_0.
template <class F>
__device__ __forceinline__ uint32_t thresholds_dev(float lam_f, F &&f) {
    const double lam = (double)lam_f;
    double p = exp(-lam);
    double Fk = p;
    uint32_t z0 = threshold_dev(Fk);
    f(0, z0);
    if (z0 == 0xFFFFFFFFu) return z0;
    for (int k = 1; k < kInvCap; ++k) {
        p = __dmul_rn(p, lam);
        p = __ddiv_rn(p, (double)k);
        Fk = __dadd_rn(Fk, p);
        const uint32_t t = threshold_dev(Fk);
        f(k, t);
        if (t == 0xFFFFFFFFu) break;
    }
    return z0;
}

// Per point: class (0 none, 1 inversion, 2 transformed rejection), tail length, lambda.
struct PointCls {
    int cls;
    uint32_t z0, z1, tail;
};

__device__ __forceinline__ PointCls classify(const PointIn &p) {
    PointCls c{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u};
    if (!p.valid || !(p.lam > 0.0f)) return c;
    if (p.lam >= kPtrsThreshold) {
        c.cls = 2;
        return c;
    }
    bool sat = false;
    uint32_t z1 = 0xFFFFFFFFu, tail = 0u;
    const uint32_t z0 = thresholds_dev(p.lam, [&](int k, uint32_t z) {
        if (k == 1) z1 = z;
        if (k >= 2 && !sat) {
            if (z == 0xFFFFFFFFu) sat = true;
            else ++tail;
        }
    });
    if (z0 == 0xFFFFFFFFu) return c;
    c.cls = 1;
    c.z0 = z0;
    c.z1 = z1;
    c.tail = tail;
    return c;
}

// Exclusive prefix sum of v over the 16 lanes of a group, and the group total.
__device__ __forceinline__ uint32_t group_scan(uint32_t v, int j, uint32_t &total) {
    uint32_t s = v;
#pragma unroll
    for (int o = 1; o < kGroup; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, s, o, kGroup);
        if (j >= o) s += u;
    }
    total = __shfl_sync(0xffffffffu, s, kGroup - 1, kGroup);
    return s - v;
}

__global__ void __launch_bounds__(256) tab_count_kernel(const TabArgs a) {
    const int h = blockIdx.y, s = blockIdx.z;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t g = t / (uint32_t)kGroup;
    const int j = (int)(t % (uint32_t)kGroup);
    const TabSetIn in = a.sets[s];
    const PointIn p = g < a.G ? point_of(a, in, g, j, h) : PointIn{0.0f, 0u, false};
    const PointCls c = classify(p);
    uint32_t n_tail, n_ptrs;
    group_scan(c.cls == 1 ? c.tail : 0u, j, n_tail);
    group_scan(c.cls == 2 ? 1u : 0u, j, n_ptrs);
    // dense: an inversion slot at or above kDenseLam
    const uint32_t act = __ballot_sync(0xffffffffu, c.cls == 1) >> (threadIdx.x & 16u) & 0xFFFFu;
    const uint32_t dense = __ballot_sync(0xffffffffu, c.cls == 1 && p.lam >= kDenseLam) >> (threadIdx.x & 16u) & 0xFFFFu;
    if (j == 0 && g < a.G) {
        const uint32_t cls = act == 0u ? 0u : (dense ? 2u : 1u);
        a.scratch[((size_t)s * 2 + h) * a.G + g] = make_uint4(cls, n_tail, n_ptrs, 0u);
    }
}

// Block-wide exclusive scan of 4 counters, 1024 threads.
__device__ __forceinline__ uint4 block_scan4(uint4 v, uint4 &total, uint4 *ws) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint4 s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, s.x, o), y = __shfl_up_sync(0xffffffffu, s.y, o);
        const uint32_t z = __shfl_up_sync(0xffffffffu, s.z, o), q = __shfl_up_sync(0xffffffffu, s.w, o);
        if (lane >= o) {
            s.x += x;
            s.y += y;
            s.z += z;
            s.w += q;
        }
    }
    if (lane == 31) ws[w] = s;
    __syncthreads();
    if (w == 0) {
        uint4 u = lane < (int)(blockDim.x >> 5) ? ws[lane] : make_uint4(0, 0, 0, 0);
        const uint4 u0 = u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, u.x, o), y = __shfl_up_sync(0xffffffffu, u.y, o);
            const uint32_t z = __shfl_up_sync(0xffffffffu, u.z, o), q = __shfl_up_sync(0xffffffffu, u.w, o);
            if (lane >= o) {
                u.x += x;
                u.y += y;
                u.z += z;
                u.w += q;
            }
        }
        ws[lane] = make_uint4(u.x - u0.x, u.y - u0.y, u.z - u0.z, u.w - u0.w);   // exclusive per warp
        if (lane == 31) ws[32] = u;
    }
    __syncthreads();
    const uint4 base = ws[w];
    total = ws[32];
    const uint4 r = make_uint4(base.x + s.x - v.x, base.y + s.y - v.y, base.z + s.z - v.z, base.w + s.w - v.w);
    __syncthreads();
    return r;
}

// Per model and half: positions of the group records (sparse list, dense list), tail offsets
// and transformed-rejection offsets, in group order; the list lengths go to the descriptor.
__global__ void __launch_bounds__(1024) tab_scan_kernel(const TabArgs a) {
    __shared__ uint4 ws[33];
    const int h = blockIdx.x, s = blockIdx.y;
    uint4 *sc = a.scratch + ((size_t)s * 2 + h) * a.G;
    uint4 carry = make_uint4(0, 0, 0, 0);
    for (uint32_t g0 = 0; g0 < a.G; g0 += blockDim.x) {
        const uint32_t g = g0 + threadIdx.x;
        const uint4 c = g < a.G ? sc[g] : make_uint4(0, 0, 0, 0);
        const uint4 v = make_uint4(c.x == 1u ? 1u : 0u, c.x == 2u ? 1u : 0u, c.y, c.z);
        uint4 tot;
        const uint4 e = block_scan4(v, tot, ws);
        if (g < a.G) {
            const uint32_t idx = c.x == 2u ? carry.y + e.y : carry.x + e.x;
            sc[g] = make_uint4(c.x, idx, carry.z + e.z, carry.w + e.w);
        }
        carry.x += tot.x;
        carry.y += tot.y;
        carry.z += tot.z;
        carry.w += tot.w;
    }
    if (threadIdx.x == 0) {
        SetDesc *d = a.desc + s;
        d->n_grp[h] = carry.x;
        d->n_dense[h] = carry.y;
        d->n_ptrs[h] = carry.w;
    }
}

__global__ void __launch_bounds__(256) tab_write_kernel(const TabArgs a) {
    const int h = blockIdx.y, s = blockIdx.z;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t g = t / (uint32_t)kGroup;
    const int j = (int)(t % (uint32_t)kGroup);
    const bool in_range = g < a.G;
    const TabSetIn in = a.sets[s];
    const PointIn p = in_range ? point_of(a, in, g, j, h) : PointIn{0.0f, 0u, false};
    const uint4 sc = in_range ? a.scratch[((size_t)s * 2 + h) * a.G + g] : make_uint4(0, 0, 0, 0);
    uint8_t *tab = a.tables + in.base;
    const TabLayout &L = a.layout;
    const int B = a.n_bands;

    // tail thresholds and slow record
    uint32_t z0 = 0xFFFFFFFFu, z1 = 0xFFFFFFFFu, len = 0u;
    const bool inv = p.valid && p.lam > 0.0f && p.lam < kPtrsThreshold;
    // this lane's tail length first (for the in-group offsets), then the values
    const PointCls c = inv ? classify(p) : PointCls{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u};
    uint32_t tot;
    const uint32_t my_tail = group_scan(c.cls == 1 ? c.tail : 0u, j, tot);
    const uint32_t my_ptrs = group_scan(p.valid && p.lam >= kPtrsThreshold ? 1u : 0u, j, tot);
    const uint32_t tail_off = (uint32_t)h * a.P * (uint32_t)(kInvCap - 2) + sc.z + my_tail;
    uint32_t *tail = reinterpret_cast<uint32_t *>(tab + L.tail_off) + tail_off;
    if (c.cls == 1) {
        z0 = c.z0;
        z1 = c.z1;
        len = c.tail;
        bool sat = false;
        uint32_t n = 0;
        thresholds_dev(p.lam, [&](int k, uint32_t z) {
            if (k >= 2 && !sat) {
                if (z == 0xFFFFFFFFu) sat = true;
                else tail[n++] = z;
            }
        });
    }
    if (in_range) {
        uint32_t ks = (uint32_t)p.lam;
        if (ks > len + 1u) ks = len + 1u;
        if (ks < 2u) ks = 2u;
        const uint4 sr = c.cls == 1 ? make_uint4(z0, z1, tail_off, len | (ks << 16))
                                    : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u);
        reinterpret_cast<uint4 *>(tab + L.slow_off[h])[(size_t)g * kGroup + j] = sr;
    }

    // fluxes of this point
    float fl[kMaxBands] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (p.valid) {
#pragma unroll
        for (int b = 0; b < kMaxBands; ++b)
            if (b < B) fl[b] = (float)__dmul_rn(a.base_flux[(size_t)p.i * B + b], in.flux_factor);
    }

    // transformed-rejection record
    if (p.valid && p.lam >= kPtrsThreshold) {
        const double lam = (double)p.lam;
        const double slam = __dsqrt_rn(lam);
        const double bb = __dadd_rn(0.931, __dmul_rn(2.53, slam));
        const double aa = __dadd_rn(-0.059, __dmul_rn(0.02483, bb));
        const double inv_alpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dsub_rn(bb, 3.4)));
        const double vr = __dsub_rn(0.9277, __ddiv_rn(3.6224, __dsub_rn(bb, 2.0)));
        PtrsRec r;
        r.i = p.i;
        r.lam = p.lam;
        r.b = (float)bb;
        r.a = (float)aa;
        r.twoa = (float)__dmul_rn(2.0, aa);
        r.vr = (float)vr;
        r.log_ia = (float)log(inv_alpha);
#pragma unroll
        for (int b = 0; b < kMaxBands; ++b) r.flux[b] = fl[b];
        r.pad = 0u;
        PtrsRec *dst = reinterpret_cast<PtrsRec *>(tab + L.ptrs_off[h]) + sc.w + my_ptrs;
        const uint4 *src4 = reinterpret_cast<const uint4 *>(&r);
        uint4 *dst4 = reinterpret_cast<uint4 *>(dst);
        dst4[0] = src4[0];
        dst4[1] = src4[1];
        dst4[2] = src4[2];
    }

    // group record (every lane writes its slot; lane 0 the header)
    if (in_range && sc.x != 0u) {
        const uint32_t rec = group_rec_bytes(B);
        uint8_t *r = tab + (sc.x == 2u ? L.dense_off[h] : L.grp_off[h]) + (size_t)sc.y * rec;
        const uint32_t zc0 = c.cls == 1 ? (z0 >> 24) : 0xFFu;
        const uint32_t zc1 = c.cls == 1 ? (z1 >> 24) : 0xFFu;
        if (j == 0) *reinterpret_cast<uint4 *>(r) = make_uint4(g, 0u, 0u, 0u);
        r[kRecZ7 + j] = (uint8_t)(zc0 & 0x7Fu);
        r[kRecZh + j] = (uint8_t)(zc0 & 0x80u);
        r[kRecZc1 + j] = (uint8_t)zc1;
        float *f = reinterpret_cast<float *>(r + kRecFlux) + j * B;
        for (int b = 0; b < B; ++b) f[b] = fl[b];
    }

    // per-point fluxes (the total-count sampler reads them by point index)
    if (p.valid && h == 0) {
        float *fo = reinterpret_cast<float *>(tab + L.flux_off) + (size_t)p.i * B;
        for (int b = 0; b < B; ++b) fo[b] = fl[b];
    }

    // inspection copies (parity export)
    if (a.insp_lam && p.valid && s == 0) {
        a.insp_lam[(size_t)h * a.P + p.i] = p.lam;
        a.insp_z0[(size_t)h * a.P + p.i] = inv ? c.z0 : 0xFFFFFFFFu;
        if (h == 0)
            for (int b = 0; b < B; ++b) a.insp_flux[(size_t)p.i * B + b] = fl[b];
    }
}

}  // namespace

TabLayout tab_layout(uint32_t P, int n_bands) {
    TabLayout L;
    const uint32_t G = (P + kGroup - 1u) / kGroup;
    const uint64_t rec = group_rec_bytes(n_bands);
    uint64_t off = 0;
    auto place = [&](uint64_t bytes) {
        const uint64_t o = off;
        off = (off + bytes + 255u) & ~uint64_t(255);
        return o;
    };
    for (int h = 0; h < 2; ++h) {
        L.grp_off[h] = place(G * rec);
        L.dense_off[h] = place(G * rec);
        L.slow_off[h] = place((uint64_t)G * kGroup * sizeof(SlowRec));
        L.ptrs_off[h] = place((uint64_t)P * sizeof(PtrsRec));
    }
    L.tail_off = place(2ull * P * (kInvCap - 2) * 4u + 4u);
    L.flux_off = place((uint64_t)P * n_bands * 4u);
    for (int h = 0; h < 2; ++h) L.pool_off[h] = place(pool_region_bytes(P));
    L.bytes = off;
    return L;
}

cudaError_t launch_build_tables(const TabArgs &a, int n_sets, cudaStream_t st) {
    if (a.G == 0 || n_sets < 1 || n_sets > 65535) return cudaErrorInvalidValue;
    const dim3 grid((a.G * kGroup + 255u) / 256u, 2, n_sets);
    tab_count_kernel<<<grid, 256, 0, st>>>(a);
    tab_scan_kernel<<<dim3(2, n_sets), 1024, 0, st>>>(a);
    tab_write_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace pcmd
