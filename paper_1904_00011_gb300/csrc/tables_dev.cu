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

// Z = ceil(F 2^32 - 1/2) - 1, saturated at 2^32 - 1; -1 when F 2^32 <= 1/2 (every word exceeds it).
__device__ __forceinline__ int64_t threshold_dev(double F) {
    const double y = __dsub_rn(__dmul_rn(F, 4294967296.0), 0.5);
    if (y >= 4294967295.0) return 0xFFFFFFFFll;
    if (!(y > 0.0)) return -1;
    const uint64_t t = (uint64_t)y;
    const uint64_t T = t + (y > (double)t ? 1u : 0u);
    return (int64_t)T - 1;
}

// IMF weight and electrons per star (distance modulus 0) of point i: the context's arrays,
// except in the grid slot an M1 model's interpolated isochrone replaces.
__device__ __forceinline__ int m1_point(const TabArgs &a, const TabSetIn &in, uint32_t i) {
    if (in.m1_k < 0) return -1;
    const uint32_t jk = i / (uint32_t)a.n_mass;
    if ((int)(jk % (uint32_t)a.n_feh) != in.m1_k) return -1;
    return (int)(in.m1_off + (jk / (uint32_t)a.n_feh) * (uint32_t)a.n_mass + i % (uint32_t)a.n_mass);
}
__device__ __forceinline__ double imf_of(const TabArgs &a, const TabSetIn &in, uint32_t i) {
    const int q = m1_point(a, in, i);
    return q < 0 ? a.imf[i] : a.m1_imf[q];
}
__device__ __forceinline__ double base_flux_of(const TabArgs &a, const TabSetIn &in, uint32_t i, int b) {
    const int q = m1_point(a, in, i);
    return q < 0 ? a.base_flux[(size_t)i * a.n_bands + b] : a.m1_flux[(size_t)q * a.n_bands + b];
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
        const double lam = __dmul_rn(w, imf_of(a, in, p.i));
        p.lam = (float)__dmul_rn(lam, a.hf[h]);
    }
    return p;
}

// Thresholds of an inversion point.  The first n0 thresholds are -1 (every word exceeds them;
// only at means above ~22, where e^-lambda 2^32 < 1/2); the count is n0 plus the walk over the
// others, Z'_k = Z_{n0 + k}.  Calls f(k, Z'_k) for k = 0 .. while Z'_k < 2^32 - 1 (and the first
// saturated one), kInvCap thresholds in all; returns n0 and Z'_0.
struct ZHead {
    uint32_t n0, z0;
};
template <class F>
__device__ __forceinline__ ZHead thresholds_dev(float lam_f, F &&f) {
    const double lam = (double)lam_f;
    double p = exp(-lam);
    double Fk = p;
    ZHead h{0u, 0xFFFFFFFFu};
    bool first = true;
    for (int k = 0; k < kInvCap; ++k) {
        if (k > 0) {
            p = __dmul_rn(p, lam);
            p = __ddiv_rn(p, (double)k);
            Fk = __dadd_rn(Fk, p);
        }
        const int64_t t = threshold_dev(Fk);
        if (t < 0) {
            h.n0 = (uint32_t)k + 1u;
            continue;
        }
        if (first) {
            h.z0 = (uint32_t)t;
            first = false;
        }
        f(k - (int)h.n0, (uint32_t)t);
        if (t == 0xFFFFFFFFll) break;
    }
    return h;
}

// Transformed-rejection record of one Poisson mean (constants of the setup in FP64, stored FP32).
__device__ __forceinline__ PtrsRec ptrs_record(float lam_f, uint32_t i, const float *fl, int nfl) {
    const double lam = (double)lam_f;
    const double slam = __dsqrt_rn(lam);
    const double bb = __dadd_rn(0.931, __dmul_rn(2.53, slam));
    const double aa = __dadd_rn(-0.059, __dmul_rn(0.02483, bb));
    const double inv_alpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dsub_rn(bb, 3.4)));
    const double vr = __dsub_rn(0.9277, __ddiv_rn(3.6224, __dsub_rn(bb, 2.0)));
    PtrsRec r;
    r.i = i;
    r.lam = lam_f;
    r.b = (float)bb;
    r.a = (float)aa;
    r.twoa = (float)__dmul_rn(2.0, aa);
    r.vr = (float)vr;
    r.log_ia = (float)log(inv_alpha);
#pragma unroll
    for (int b = 0; b < kMaxBands; ++b) r.flux[b] = b < nfl ? fl[b] : 0.0f;
    r.pad = 0u;
    return r;
}

// Per point: class (0 none, 1 inversion, 2 transformed rejection), leading count n0, the first
// two thresholds after it and the tail length.
struct PointCls {
    int cls;
    uint32_t z0, z1, tail, n0, nw;
};

// The one pass over the threshold series: Z'_0, Z'_1, ... (up to the first saturated one, at most
// kTailCap) go to `slot`, the point's fixed slot of kTailCap words; nw counts the words written.
__device__ __forceinline__ PointCls classify(const PointIn &p, uint32_t *slot) {
    PointCls c{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u, 0u};
    if (!p.valid || !(p.lam > 0.0f)) return c;
    if (p.lam >= kPtrsThreshold) {
        c.cls = 2;
        return c;
    }
    bool sat = false;
    uint32_t z1 = 0xFFFFFFFFu, tail = 0u, nw = 0u;
    const ZHead zh = thresholds_dev(p.lam, [&](int k, uint32_t z) {
        if (k == 1) z1 = z;
        if (nw < (uint32_t)kTailCap) slot[nw++] = z;    // k = nw: Z'_k at word k (the cap is unreachable below 640)
        if (k >= 2 && !sat) {
            if (z == 0xFFFFFFFFu) sat = true;
            else ++tail;
        }
    });
    c.nw = nw;
    if (zh.n0 == 0u && zh.z0 == 0xFFFFFFFFu) return c;    // never a star
    c.cls = 1;
    c.z0 = zh.z0;
    c.z1 = z1;
    c.tail = tail;
    c.n0 = zh.n0;
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

// Total-count sampler weights in fixed point: L = floor(lambda 2^40) for 0 < lambda < 640 (exact:
// lambda 2^40 is exact in FP64), 0 otherwise; a point is in the pool when L > 0.
__device__ __forceinline__ uint64_t pool_weight(const PointIn &p) {
    if (!p.valid || !(p.lam > 0.0f) || !(p.lam < kPtrsThreshold)) return 0ull;
    return __double2ull_rz(__dmul_rn((double)p.lam, kPoolFix));
}

// Inclusive prefix sum of a 64-bit value over the 16 lanes of a group, and the group total.
__device__ __forceinline__ uint64_t group_scan64(uint64_t v, int j, uint64_t &total) {
    uint64_t s = v;
#pragma unroll
    for (int o = 1; o < kGroup; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, s, o, kGroup);
        if (j >= o) s += u;
    }
    total = __shfl_sync(0xffffffffu, s, kGroup - 1, kGroup);
    return s;
}

// T = min(floor(C 2^32 / L), 2^32 - 1) for 0 <= C <= L, L > 0, exactly: an FP64 estimate (off
// by less than 2), corrected against the exact 128-bit products.
__device__ __forceinline__ uint32_t pool_threshold(uint64_t C, uint64_t L) {
    const double e = floor(__dmul_rn(__ddiv_rn(__ull2double_rn(C), __ull2double_rn(L)), 4294967296.0));
    uint64_t q = (uint64_t)e;
    const unsigned __int128 num = (unsigned __int128)C << 32;
    unsigned __int128 m = (unsigned __int128)q * L;
    for (int it = 0; it < 4 && m > num; ++it) {
        --q;
        m -= L;
    }
    for (int it = 0; it < 4 && num - m >= L; ++it) {
        ++q;
        m += L;
    }
    return q >= 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)q;
}

__device__ __forceinline__ uint4 *pool_scratch(const TabArgs &a, int s, int h) {
    return a.pool_scratch + ((size_t)s * 2 + h) * a.G;
}

__global__ void __launch_bounds__(256) tab_count_kernel(const TabArgs a) {
    const int h = blockIdx.y, s = blockIdx.z;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t g = t / (uint32_t)kGroup;
    const int j = (int)(t % (uint32_t)kGroup);
    const TabSetIn in = a.sets[s];
    const PointIn p = g < a.G ? point_of(a, in, g, j, h) : PointIn{0.0f, 0u, false};
    // thresholds of point slot t of half h: a fixed slot of kTailCap words
    uint32_t *tail = reinterpret_cast<uint32_t *>(a.tables + in.base + a.layout.tail_off) +
                     ((size_t)h * a.G * kGroup + t) * kTailCap;
    const PointCls c = classify(p, tail);
    if (g < a.G)   // the write pass reads these instead of running the threshold series again
        a.pt_scratch[((size_t)s * 2 + h) * a.G * kGroup + t] = make_uint4(c.z0, c.z1, c.tail, (uint32_t)c.cls | (c.n0 << 8));
    uint32_t n_tail, n_ptrs;
    group_scan(c.cls == 1 ? c.tail : 0u, j, n_tail);
    group_scan(c.cls == 2 ? 1u : 0u, j, n_ptrs);
    // dense: an inversion slot at or above kDenseLam
    const uint32_t act = __ballot_sync(0xffffffffu, c.cls == 1) >> (threadIdx.x & 16u) & 0xFFFFu;
    const uint32_t dense = __ballot_sync(0xffffffffu, c.cls == 1 && p.lam >= kDenseLam) >> (threadIdx.x & 16u) & 0xFFFFu;
    // the slots of a dense group's inversion points are saturated (2^32 - 1) to their end, so that
    // a walk through them needs no length
    if (dense && c.cls == 1)
        for (uint32_t k = c.nw; k < (uint32_t)kTailCap; ++k) tail[k] = 0xFFFFFFFFu;
    if (j == 0 && g < a.G) {
        const uint32_t cls = act == 0u ? 0u : (dense ? 2u : 1u);
        a.scratch[((size_t)s * 2 + h) * a.G + g] = make_uint4(cls, n_tail, n_ptrs, 0u);
    }
    if (a.pool) {
        const uint64_t wq = pool_weight(p);
        const uint32_t n = __popc(__ballot_sync(0xffffffffu, wq > 0ull) >> (threadIdx.x & 16u) & 0xFFFFu);
        uint64_t sum;
        group_scan64(wq, j, sum);
        if (j == 0 && g < a.G) pool_scratch(a, s, h)[g] = make_uint4(n, (uint32_t)sum, (uint32_t)(sum >> 32), 0u);
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

// Block-wide exclusive scan of a 64-bit value, 1024 threads.
__device__ __forceinline__ uint64_t block_scan64(uint64_t v, uint64_t &total, uint64_t *ws) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t x = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += x;
    }
    if (lane == 31) ws[w] = s;
    __syncthreads();
    if (w == 0) {
        uint64_t u = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0ull;
        const uint64_t u0 = u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t x = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += x;
        }
        ws[lane] = u - u0;
        if (lane == 31) ws[32] = u;
    }
    __syncthreads();
    const uint64_t r = ws[w] + s - v;
    total = ws[32];
    __syncthreads();
    return r;
}

// Header of a total-count sampler region: pool size n, Lambda = (float)(Lfix 2^-40) (the FP64
// conversion rounds to nearest), the draw of the total (inversion thresholds below 10, a
// transformed-rejection record at and above), and the fixed-point total itself.
__device__ void write_pool_header(uint8_t *pr, uint32_t P, uint32_t n, uint64_t lfix) {
    *reinterpret_cast<uint64_t *>(pr + pool_fix_off(P)) = lfix;
    PoolHdr hdr{0.0f, n, 0u, 0u};
    if (n > 0) {
        hdr.lam = __double2float_rn(__dmul_rn(__ull2double_rn(lfix), 1.0 / kPoolFix));
        if (hdr.lam < kPoolTotalLimit) {
            uint32_t *z = reinterpret_cast<uint32_t *>(pr + kPoolZOff);
            const ZHead zh = thresholds_dev(hdr.lam, [&](int k, uint32_t zk) {
                z[k] = zk;
                hdr.n_z = (uint32_t)k + 1u;
            });
            hdr.mode = 1u | (zh.n0 << 8);       // the total is n0 + #{k : x > z[k]}
        } else {
            hdr.mode = 2u;
            *reinterpret_cast<PtrsRec *>(pr + kPoolPtrsOff) = ptrs_record(hdr.lam, 0xFFFFFFFFu, nullptr, 0);
        }
    }
    *reinterpret_cast<PoolHdr *>(pr) = hdr;
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
        // the word tables have room for btab_cap dense groups per half (an upper bound from the
        // host's FP64 lambda bound): more is an internal error, latched, and the list is cut so
        // that nothing reads or writes past the tables
        uint32_t nd = carry.y;
        if (a.btab && nd > d->btab_cap) {
            atomicOr(a.err, kErrBounds);
            nd = d->btab_cap;
        }
        d->n_dense[h] = nd;
        d->n_ptrs[h] = carry.w;
    }
    if (!a.pool) return;
    // total-count sampler: pool positions and fixed-point cumulative sums of every group
    __shared__ uint64_t ws64[33];
    uint4 *ps = pool_scratch(a, s, h);
    uint32_t pn = 0;
    uint64_t pc = 0;
    for (uint32_t g0 = 0; g0 < a.G; g0 += blockDim.x) {
        const uint32_t g = g0 + threadIdx.x;
        const uint4 c = g < a.G ? ps[g] : make_uint4(0, 0, 0, 0);
        uint4 tot;
        const uint4 e = block_scan4(make_uint4(c.x, 0, 0, 0), tot, ws);
        uint64_t tot64;
        const uint64_t e64 = block_scan64((uint64_t)c.y | (uint64_t)c.z << 32, tot64, ws64);
        if (g < a.G) {
            const uint64_t base = pc + e64;
            ps[g] = make_uint4(pn + e.x, (uint32_t)base, (uint32_t)(base >> 32), 0u);
        }
        pn += tot.x;
        pc += tot64;
    }
    if (threadIdx.x == 0) write_pool_header(a.tables + a.sets[s].base + a.layout.pool_off[h], a.P, pn, pc);
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
    PointCls c{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u};
    if (inv) {   // as the count pass classified it
        const uint4 pc = a.pt_scratch[((size_t)s * 2 + h) * a.G * kGroup + t];
        c.z0 = pc.x;
        c.z1 = pc.y;
        c.tail = pc.z;
        c.cls = (int)(pc.w & 0xFFu);
        c.n0 = pc.w >> 8;
    }
    uint32_t tot;
    const uint32_t my_ptrs = group_scan(p.valid && p.lam >= kPtrsThreshold ? 1u : 0u, j, tot);
    // a dense group with an inversion mean of kWideLam or more takes the wide word-table layout
    const uint32_t wide = __ballot_sync(0xffffffffu, inv && p.lam >= kWideLam) >> (threadIdx.x & 16u) & 0xFFFFu;
    // the count pass wrote Z'_0, Z'_1, ... into the point's fixed slot; the slow record's tail offset
    // points at Z'_2
    const uint32_t tail_off = (uint32_t)(((size_t)h * a.G * kGroup + t) * kTailCap) + 2u;
    if (c.cls == 1) {
        z0 = c.z0;
        z1 = c.z1;
        len = c.tail;
    }
    if (in_range) {
        // the walk starts near the mean, in the shifted sequence Z'_k = Z_{n0 + k}
        const uint32_t lk = (uint32_t)p.lam;
        uint32_t ks = lk > c.n0 ? lk - c.n0 : 0u;
        if (ks > len + 1u) ks = len + 1u;
        if (ks < 2u) ks = 2u;
        const uint4 sr = c.cls == 1 ? make_uint4(z0, z1, tail_off, slow_pack(len, c.n0, ks))
                                    : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u);
        reinterpret_cast<uint4 *>(tab + L.slow_off[h])[(size_t)g * kGroup + j] = sr;
    }

    // fluxes of this point
    float fl[kMaxBands] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (p.valid) {
#pragma unroll
        for (int b = 0; b < kMaxBands; ++b)
            if (b < B) fl[b] = (float)__dmul_rn(base_flux_of(a, in, p.i, b), in.flux_factor);
    }

    // transformed-rejection record
    if (p.valid && p.lam >= kPtrsThreshold) {
        const PtrsRec r = ptrs_record(p.lam, p.i, fl, kMaxBands);
        PtrsRec *dst = reinterpret_cast<PtrsRec *>(tab + L.ptrs_off[h]) + sc.w + my_ptrs;
        const uint4 *src4 = reinterpret_cast<const uint4 *>(&r);
        uint4 *dst4 = reinterpret_cast<uint4 *>(dst);
        dst4[0] = src4[0];
        dst4[1] = src4[1];
        dst4[2] = src4[2];
    }

    // group record (every lane writes its slot; lane 0 the header)
    if (in_range && sc.x != 0u) {
        const uint32_t rec = sc.x == 2u ? group_rec_bytes(B) : kSparseRecBytes;
        uint8_t *r = tab + (sc.x == 2u ? L.dense_off[h] : L.grp_off[h]) + (size_t)sc.y * rec;
        const uint32_t zc0 = c.cls == 1 ? (z0 >> 24) : 0xFFu;
        const uint32_t zc1 = c.cls == 1 ? (z1 >> 24) : 0xFFu;
        if (j == 0) *reinterpret_cast<uint4 *>(r) = make_uint4(g, sc.x == 2u && wide ? 1u : 0u, 0u, 0u);
        // a dense record keeps each slot's leading count n0 (u16) where a sparse one has its coarse
        // bytes and their top bits
        if (sc.x == 2u) {
            reinterpret_cast<uint16_t *>(r + kRecN0)[j] = (uint16_t)(c.cls == 1 ? c.n0 : 0u);
        } else {
            r[kRecZ7 + j] = (uint8_t)(zc0 & 0x7Fu);
            r[kRecZh + j] = (uint8_t)(zc0 & 0x80u);
        }
        r[kRecZc1 + j] = (uint8_t)zc1;
        if (sc.x == 2u) {   // dense records carry their fluxes (sparse ones use the flux table)
            float *f = reinterpret_cast<float *>(r + kRecFlux) + j * B;
            for (int b = 0; b < B; ++b) f[b] = fl[b];
        }
    }

    // total-count sampler: this point's pool entry (point index, star-assignment threshold)
    if (a.pool) {
        const uint64_t wq = in_range ? pool_weight(p) : 0ull;
        uint32_t n_in_group;
        const uint32_t my_pos = group_scan(wq > 0ull ? 1u : 0u, j, n_in_group);
        uint64_t w_in_group;
        const uint64_t my_c = group_scan64(wq, j, w_in_group);
        if (wq > 0ull) {
            uint8_t *pr = tab + L.pool_off[h];
            const uint4 ps = pool_scratch(a, s, h)[g];
            const uint32_t n = reinterpret_cast<const PoolHdr *>(pr)->n;
            const uint64_t lfix = *reinterpret_cast<const uint64_t *>(pr + pool_fix_off(a.P));
            const uint64_t C = ((uint64_t)ps.y | (uint64_t)ps.z << 32) + my_c;
            uint32_t *idx = reinterpret_cast<uint32_t *>(pr + kPoolIdxOff);
            idx[ps.x + my_pos] = p.i;
            idx[n + ps.x + my_pos] = pool_threshold(C, lfix);
        }
    }

    // per-point fluxes (the total-count sampler reads them by point index)
    if (p.valid && h == 0) {
        float *fo = reinterpret_cast<float *>(tab + L.flux_off) + (size_t)p.i * B;
        for (int b = 0; b < B; ++b) fo[b] = fl[b];
    }

    // inspection copies (parity export)
    if (a.insp_lam && p.valid && s == 0) {
        a.insp_lam[(size_t)h * a.P + p.i] = p.lam;
        a.insp_z0[(size_t)h * a.P + p.i] = inv && c.n0 == 0u ? c.z0 : 0xFFFFFFFFu;
        if (h == 0)
            for (int b = 0; b < B; ++b) a.insp_flux[(size_t)p.i * B + b] = fl[b];
    }
}

// Guide table of a total-count sampler region, one thread per pool entry.
// guide[b] = first entry j < n - 1 with T_j > b 2^s (s = 32 - bits), else n - 1: entry j owns
// the buckets with T_{j-1} <= b 2^s < T_j (T_{-1} = 0); buckets at or above T_{n-2} get n - 1.
__global__ void __launch_bounds__(256) tab_pool_guide_kernel(const TabArgs a) {
    const int h = blockIdx.y, s = blockIdx.z;
    const TabSetIn in = a.sets[s];
    uint8_t *pr = a.tables + in.base + a.layout.pool_off[h];
    const uint32_t n = reinterpret_cast<const PoolHdr *>(pr)->n;
    uint32_t *guide = reinterpret_cast<uint32_t *>(pr + kPoolGuideOff);
    const uint32_t *thr = reinterpret_cast<const uint32_t *>(pr + kPoolIdxOff) + n;
    constexpr uint32_t sh = 32 - kPoolGuideBits;
    const uint32_t nbk = 1u << kPoolGuideBits;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t top = n > 1 ? ((uint64_t)thr[n - 2] + (1ull << sh) - 1) >> sh : 0;
    if (t + 1 < n) {
        const uint64_t t0 = t > 0 ? thr[t - 1] : 0u, t1 = thr[t];
        const uint64_t b0 = (t0 + (1ull << sh) - 1) >> sh;
        const uint64_t b1 = t1 > 0 ? ((t1 - 1) >> sh) + 1 : 0;
        for (uint64_t b = b0; b < b1; ++b) guide[b] = t;
    }
    if (t <= nbk && (t >= top || t == nbk)) guide[t] = n > 0 ? n - 1 : 0u;
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
        L.grp_off[h] = place(G * kSparseRecBytes);
        L.dense_off[h] = place(G * rec);
        L.slow_off[h] = place((uint64_t)G * kGroup * sizeof(SlowRec));
        L.ptrs_off[h] = place((uint64_t)P * sizeof(PtrsRec));
    }
    L.tail_off = place(2ull * ((P + kGroup - 1u) / kGroup) * kGroup * kTailCap * 4u + 4u);
    L.flux_off = place((uint64_t)P * n_bands * 4u);
    for (int h = 0; h < 2; ++h) L.pool_off[h] = place(pool_region_bytes(P));
    L.bytes = off;
    return L;
}

namespace {

// n0 + (first k with x <= Z'_k): the count of word x from a slow record, by binary search over
// the shifted thresholds (Z'_k saturated from len + 2 on).
__device__ __forceinline__ uint32_t count_bsearch(uint32_t x, const uint4 &sr, const uint32_t *tail) {
    const uint32_t n0 = slow_n0(sr.w), len = slow_len(sr.w);
    auto z = [&](uint32_t k) -> uint32_t {
        return k == 0u ? sr.x : k == 1u ? sr.y : (k - 2u < len ? tail[sr.z + (k - 2u)] : 0xFFFFFFFFu);
    };
    uint32_t lo = 0u, hi = len + 2u;                 // z(hi) = 2^32 - 1 >= x
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (x <= z(mid)) hi = mid;
        else lo = mid + 1u;
    }
    return n0 + lo;
}

// Word tables of the dense groups: one CTA per (dense-list position, half, model); 16 threads per
// slot, each for 16 consecutive HI bytes, walking the slot's thresholds alongside the byte edges
// (one binary search for the first byte, then a merge).  For byte b: c0 = count(b << 24), c1 =
// count((b << 24) | 0xFFFFFF).  One threshold or none inside the byte: c0 and Z_c0's bits inside
// the byte (all ones when c1 = c0).  Two or more (the flag): the count m in [c0, c1] that holds the
// most words of the byte and Z_m's bits (all ones when m = c1), so that most words of
// the byte end where the search starts.  Counts are stored relative to the slot's n0.
__global__ void __launch_bounds__(256) tab_btab_kernel(const TabArgs a) {
    const uint32_t q = blockIdx.x;
    const int h = blockIdx.y, s = blockIdx.z;
    const SetDesc &d = a.desc[s];
    if (q >= d.n_dense[h]) return;
    const uint32_t rec = group_rec_bytes(a.n_bands);
    const uint2 hd = *reinterpret_cast<const uint2 *>(a.tables + d.dense_off[h] + (uint64_t)q * rec);
    const uint32_t gid = hd.x;
    const bool wide = hd.y != 0u;
    const uint4 *slow = reinterpret_cast<const uint4 *>(a.tables + d.slow_off[h]) + (uint64_t)gid * kGroup;
    const uint32_t *tail = reinterpret_cast<const uint32_t *>(a.tables + d.tail_off);
    uint32_t *out = reinterpret_cast<uint32_t *>(a.btab + d.btab_off[h]) + (uint64_t)q * kBtabGroupEntries;
    for (uint32_t t = threadIdx.x; t < kGroup * 16u; t += blockDim.x) {
        const uint32_t j = t >> 4, b0 = (t & 15u) * 16u;
        const uint4 sr = slow[j];
        const uint32_t n0 = slow_n0(sr.w), len = slow_len(sr.w);
        // Z_c (c >= n0: every word exceeds the first n0 thresholds); 2^32 - 1 from len + 2 on
        auto zc = [&](uint32_t c) -> uint32_t {
            const uint32_t k = c - n0;
            return k == 0u ? sr.x : k == 1u ? sr.y : (k - 2u < len ? tail[sr.z + (k - 2u)] : 0xFFFFFFFFu);
        };
        const uint32_t cmax = n0 + (wide ? 0xFFu : 0x7Fu);   // c - n0 in 8 (wide) or 7 bits
        uint32_t cur = count_bsearch(b0 << 24, sr, tail);
        for (uint32_t b = b0; b < b0 + 16u; ++b) {
            const uint32_t lo = b << 24, hi = lo | 0xFFFFFFu;
            while (zc(cur) < lo) ++cur;                 // count(lo) = #{k : Z_k < lo}
            const uint32_t c0 = cur;
            uint32_t c1 = c0;
            while (zc(c1) < hi) ++c1;                   // count(hi)
            // the threshold's bits inside the byte: low 24 (narrow) or bits 1-23 (wide); all ones
            // when the count does not change over the byte
            const uint32_t zshift = wide ? 1u : 0u, zmask = wide ? 0x7FFFFFu : 0xFFFFFFu;
            uint32_t c = c0, zl = zmask;
            if (c1 == c0 + 1u) {
                zl = (zc(c0) >> zshift) & zmask;        // Z_c0 lies inside the byte: its top byte is b
            } else if (c1 > c0 + 1u) {
                // words of count m in the byte: [max(Z_{m-1} + 1, lo), min(Z_m, hi)] (empty when two
                // thresholds are equal)
                uint32_t best = 0u, wlo = lo;
                for (uint32_t m = c0; m <= c1 && m <= cmax; ++m) {
                    const uint32_t whi = m == c1 ? hi : zc(m);
                    const uint32_t width = whi >= wlo ? whi - wlo + 1u : 0u;
                    if (m == c0 || width > best) {
                        best = width;
                        c = m;
                    }
                    wlo = whi + 1u;
                }
                zl = c == c1 ? zmask : ((zc(c) >> zshift) & zmask);
            }
            // the count at any byte's lower edge is at most n0 + 119 below a mean of 192 (narrow)
            // and n0 + 222 below 640 (wide)
            const bool multi = c1 > c0 + 1u;
            out[j * 256u + b] = wide ? (((c - n0) & 0xFFu) | (zl << 8) | (multi ? 0x80000000u : 0u))
                                     : (((c - n0) & 0x7Fu) | (multi ? 0x80u : 0u) | (zl << 8));
            cur = c1;                                   // count((b + 1) << 24) >= count(hi)
        }
    }
}

}  // namespace

cudaError_t launch_build_tables(const TabArgs &a, int n_sets, cudaStream_t st) {
    if (a.G == 0 || n_sets < 1 || n_sets > 65535) return cudaErrorInvalidValue;
    const dim3 grid((a.G * kGroup + 255u) / 256u, 2, n_sets);
    tab_count_kernel<<<grid, 256, 0, st>>>(a);
    tab_scan_kernel<<<dim3(2, n_sets), 1024, 0, st>>>(a);
    tab_write_kernel<<<grid, 256, 0, st>>>(a);
    if (a.btab) tab_btab_kernel<<<dim3(a.G, 2, n_sets), 256, 0, st>>>(a);
    if (a.pool) {
        const uint32_t ng = (max(a.P, (1u << kPoolGuideBits) + 1) + 255) / 256;
        tab_pool_guide_kernel<<<dim3(ng, 2, n_sets), 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace pcmd
