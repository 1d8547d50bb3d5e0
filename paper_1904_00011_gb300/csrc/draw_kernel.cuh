// draw_flux: Poisson star counts per pixel and isochrone point, per-band flux sums, dust
// screen and (fused mode) noise, magnitudes and the Hess diagram.
//
// Section 2.1: every pixel receives n_i ~ Poisson(lambda_i) stars at every age-[Fe/H]-mass
// point, lambda summing to Npix; fluxes are summed per band (panels B-D of Fig. 1), the dust
// screen dims the stars behind it (Section 2.2 E1-E3) and distance is folded into the per-star
// fluxes (D1/D2).  Section 2.4: the paper gives one GPU thread per pixel; here one thread per
// pixel and split (a CTA's warps share a pixel tile and divide the isochrone points), with
// the point tables streamed through shared memory by bulk copies.
//
// Draw word of inversion point i (lambda < 640) of half h at pixel p:
//   x = b << 24 | l >> 8, b = byte i & 3 of word (i & 15) >> 2 of Philox(p, i >> 4, set, HI|h),
//   l = word i & 3 of Philox(p, i >> 2, set, LO|h);  n = #{k : x > Z_k}.
// The fast path only needs b: b < Z_0 >> 24 gives n = 0 without the LO call, and a certain hit
// with Z_0 >> 24 < b < Z_1 >> 24 gives n = 1.  Both are exact consequences of the rule.
#pragma once
#include "common.cuh"

namespace pcmd {

// stirlerr(k) for k < 16; one copy per translation unit that includes this file (each uploads
// its own copy through upload_stirlerr_local).
static __constant__ float c_stirlerr[16];

static cudaError_t upload_stirlerr_local(const float *tab16) {
    return cudaMemcpyToSymbol(c_stirlerr, tab16, 16 * sizeof(float));
}

// stirlerr(k) = ln k! - (k ln k - k + ln(2 pi k) / 2): table below 16 (built in FP64 on the
// host), FP32 Stirling series 1/(12k) - 1/(360k^3) + 1/(1260k^5) above (DLMF 5.11.1).
__device__ __forceinline__ float stirlerr_dev(float kf) {
    if (kf < 16.0f) return c_stirlerr[(int)kf];
    const float r = __fdiv_rn(1.0f, kf);
    const float r2 = __fmul_rn(r, r);
    float t = __fmul_rn(r2, (float)(1.0 / 1260.0));
    t = __fsub_rn((float)(1.0 / 360.0), t);
    t = __fmul_rn(t, r2);
    t = __fsub_rn((float)(1.0 / 12.0), t);
    return __fmul_rn(t, r);
}

// Transformed rejection with squeeze (Hormann 1993) for lambda >= 640.  Attempt `at` uses words
// 2(at&1), 2(at&1)+1 of Philox(p, i, set, PTRS|h|at>>1).  The cheap part of an attempt decides
// the squeeze acceptance and the quick rejections; the rest takes the log-form test.
struct PtrsTry {
    float kf, us, V;
    int status;   // 0 accept, 1 reject, 2 needs the log test
};

__device__ __forceinline__ PtrsTry ptrs_cheap(const PtrsRec &r, uint32_t wu, uint32_t wv) {
    PtrsTry t;
    const float U = __fsub_rn(uniform_of(wu), 0.5f);
    t.V = uniform_of(wv);
    t.us = __fsub_rn(0.5f, fabsf(U));
    float x = __fdiv_rn(r.twoa, t.us);
    x = __fadd_rn(x, r.b);
    x = __fmul_rn(x, U);
    x = __fadd_rn(x, r.lam);
    x = __fadd_rn(x, 0.43f);
    t.kf = floorf(x);
    if (t.us >= 0.07f && t.V <= r.vr) t.status = 0;
    else if (t.kf < 0.0f || (t.us < 0.013f && t.V > t.us) || t.kf > 1.0e9f) t.status = 1;
    else t.status = 2;
    return t;
}

// The log-form test: ln V + ln inv_alpha - ln q <= log pmf(k), q = a / us^2 + b.  For k >= 1
// the pmf's term -ln(k) / 2 moves to the left-hand side, which then takes one logarithm:
// ln(V sqrt(k) / q) + ln inv_alpha <= -lambda phi((k - lambda) / lambda) - ln(2 pi) / 2 -
// stirlerr(k); k = 0 keeps ln V + ln inv_alpha - ln q <= -lambda.
__device__ __forceinline__ bool ptrs_log_accept(const PtrsRec &r, const PtrsTry &t) {
    float q = __fmul_rn(t.us, t.us);
    q = __fdiv_rn(r.a, q);
    q = __fadd_rn(q, r.b);
    if (t.kf == 0.0f) {
        float lhs = ln_series(t.V);
        lhs = __fadd_rn(lhs, r.log_ia);
        lhs = __fsub_rn(lhs, ln_series(q));
        return lhs <= -r.lam;
    }
    float y = __fmul_rn(t.V, __fsqrt_rn(t.kf));
    y = __fdiv_rn(y, q);
    const float lhs = __fadd_rn(ln_series(y), r.log_ia);
    const float x = __fdiv_rn(__fsub_rn(t.kf, r.lam), r.lam);
    float rhs = -__fmul_rn(r.lam, phi_dev(x));
    rhs = __fsub_rn(rhs, (float)0.91893853320467274178);
    rhs = __fsub_rn(rhs, stirlerr_dev(t.kf));
    return lhs <= rhs;
}

__device__ __forceinline__ uint4 ptrs_words(const PtrsRec &r, uint32_t pix, uint32_t set, uint32_t half,
                                            uint32_t at, const uint32_t *rk0, const uint32_t *rk1) {
    return philox_rk(pix, r.i, set, rng_tag(kKindPtrs, half, at >> 1), rk0, rk1);
}

// The attempt loop of one draw; out of line, so that the caller's registers stay its own.
// After `cap` attempts without acceptance the draw gives 0 and latches kErrSampler.
static __device__ __noinline__ uint32_t ptrs_draw(const PtrsRec &r, uint32_t pix, uint32_t set, uint32_t half,
                                           const uint32_t *rk0, const uint32_t *rk1, uint32_t cap,
                                           uint32_t *err) {
    uint4 w = make_uint4(0, 0, 0, 0);
    for (uint32_t at = 0; at < cap; ++at) {
        if ((at & 1u) == 0u) w = ptrs_words(r, pix, set, half, at, rk0, rk1);
        const PtrsTry t = ptrs_cheap(r, (at & 1u) ? w.z : w.x, (at & 1u) ? w.w : w.y);
        if (t.status == 0) return (uint32_t)t.kf;
        if (t.status == 1) continue;
        if (ptrs_log_accept(r, t)) return (uint32_t)t.kf;
    }
    atomicOr(err, kErrSampler);
    return 0u;
}

// Per-pixel flux accumulators of the two dust halves; compensated (Kahan) when KAHAN.
template <int B, bool KAHAN>
struct Acc {
    float s[2][B];
    float c[2][B];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int b = 0; b < B; ++b) s[h][b] = c[h][b] = 0.0f;
    }
    template <int H>
    __device__ __forceinline__ void add(float n, const float *f) {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const float v = __fmul_rn(n, f[b]);
            if (KAHAN) {
                const float y = __fsub_rn(v, c[H][b]);
                const float t = __fadd_rn(s[H][b], y);
                c[H][b] = __fsub_rn(__fsub_rn(t, s[H][b]), y);
                s[H][b] = t;
            } else {
                s[H][b] = __fadd_rn(s[H][b], v);
            }
        }
    }
    template <int H>
    __device__ __forceinline__ void add_sum(const float *v) {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (KAHAN) {
                const float y = __fsub_rn(v[b], c[H][b]);
                const float t = __fadd_rn(s[H][b], y);
                c[H][b] = __fsub_rn(__fsub_rn(t, s[H][b]), y);
                s[H][b] = t;
            } else {
                s[H][b] = __fadd_rn(s[H][b], v[b]);
            }
        }
    }
    template <int H>
    __device__ __forceinline__ float value(int b) const {
        return KAHAN ? __fsub_rn(s[H][b], c[H][b]) : s[H][b];
    }
};

// "Maybe non-zero" bits of the 16 slots of one HI call: bit 7 of byte j & 3 of word j >> 2 is
// set iff HI byte j >= zc_j.  Per byte, (x | 0x80) - (zc & 0x7F) has bit 7 iff the low seven
// bits of x are >= those of zc (no borrow leaves the byte); the top bits decide the rest.
__device__ __forceinline__ uint32_t ge_bytes(uint32_t x, uint32_t z7, uint32_t zh) {
    const uint32_t d = (x | 0x80808080u) - z7;
    return (x & ~zh) | (~(x ^ zh) & d);          // bit 7 of each byte; other bits are noise
}

struct ItemCtx {
    uint32_t pix, set, npix;
    bool active;
    const SlowRec *slow[2];
    const uint32_t *tail;
    const float *flux;      // [P][B] electrons per star of every point
};

constexpr int kQueueCap = 16;   // hit-queue entries per thread (shared memory)

// The chunk double buffer: two chunks of group records.
__host__ __device__ constexpr uint32_t chunk_region_bytes(uint32_t chunk, uint32_t rec) { return 2u * chunk * rec; }

// n = #{k : x > Z_k} from the slow record of a slot: the first n0 thresholds are -1 (every word
// exceeds them), Z'_k = Z_{n0 + k}: Z'_0, Z'_1 in the record, Z'_2.. in the tail (saturated
// beyond its length).  n = n0 + #{k : x > Z'_k}.  The search starts at the record's start index
// k_s (near lambda - n0) and walks up or down; the count equals the linear scan's.
__device__ __forceinline__ uint32_t count_from_thresholds(uint32_t x, const uint4 &sr, const uint32_t *tail) {
    const uint32_t n0 = slow_n0(sr.w);
    if (x <= sr.x) return n0;
    if (x <= sr.y) return n0 + 1u;
    const uint32_t len = slow_len(sr.w);
    uint32_t ks = slow_ks(sr.w);                    // 2 <= ks <= len + 1
    if (ks < 2u) ks = 2u;
    auto z = [&](uint32_t k) { return k - 2u < len ? __ldg(tail + sr.z + (k - 2u)) : 0xFFFFFFFFu; };
    uint32_t k = ks;
    if (x > z(k)) {
        do { ++k; } while (k - 2u < len && x > z(k));
        return n0 + k;                              // first k with x <= Z'_k
    }
    while (k > 2u && x <= z(k - 1u)) --k;
    return n0 + k;
}

// Walks over a dense slot's thresholds zs (zs[k] = Z_{n0 + k}, saturated to the slot's end), in
// counts relative to n0: upwards, the first k >= k0 with x <= zs[k] (given x > zs[k0 - 1]);
// downwards, the last k <= k0 with x > zs[k - 1], or 0 (given x <= zs[k0]).
__device__ __forceinline__ uint32_t slot_up(uint32_t x, const uint32_t *zs, uint32_t k) {
    while (k < (uint32_t)kTailCap - 1u && x > __ldg(zs + k)) ++k;
    return k;
}
__device__ __forceinline__ uint32_t slot_down(uint32_t x, const uint32_t *zs, uint32_t k) {
    while (k > 0u && x <= __ldg(zs + k - 1u)) --k;
    return k;
}

// The warp's queued maybe-hits, resolved by all 32 lanes together.  Queue entry of a lane's
// group with maybe-hits: g | prefix << 8 | hm << 16, g the group's index in the staged chunk,
// hm its maybe-hit mask (bit 4q + k = byte q of HI word k = slot 4k + q), prefix the number of
// maybe-hit bits in the lane's earlier entries (written here).  The bits of all 32 lanes are
// enumerated as one list (lane order, then entry order, then bit order); every lane takes every
// 32nd: it finds the owner lane and entry by binary searches, recomputes the owner's HI word,
// and decides n: 1 when the byte is above Z_0 >> 24 and below Z_1 >> 24, otherwise the LO call
// of the slot's quad completes the 32-bit word and the full thresholds decide.  The fluxes
// n f_b of one owner's consecutive list positions are summed by a segmented warp scan (a fixed
// tree), each owner adds its segments' totals in list order, and the drain's total goes into
// the pixel's accumulator once.  Called by all 32 lanes of the warp.
template <int B, bool KAHAN, int MODE, int H>
__device__ __forceinline__ void drain_warp(const DrawArgs &a, const ItemCtx &ic, const PhiloxPrefix &pf,
                                           const uint8_t *cb, uint32_t *queue, int qn,
                                           Acc<B, KAHAN> &acc) {
    constexpr uint32_t rec = kSparseRecBytes;
    const uint32_t lane = threadIdx.x & 31u, wbase = threadIdx.x & ~31u, bd = blockDim.x;
    uint32_t nb = 0;
    for (int e = 0; e < qn; ++e) {
        uint32_t *q = queue + (uint32_t)e * bd + threadIdx.x;
        const uint32_t m = *q;
        *q = (m & 0xFFFF00FFu) | (nb << 8);
        nb += (uint32_t)__popc(m >> 16);
    }
    uint32_t inc = nb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    const uint32_t off = inc - nb;                      // first list position of this lane's bits
    float part[B];
#pragma unroll
    for (int b = 0; b < B; ++b) part[b] = 0.0f;
    for (uint32_t v0 = 0; v0 < total; v0 += 32u) {
        const uint32_t v = v0 + lane;
        uint32_t o = 0;                                  // owner: last lane with off <= v
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const uint32_t t = __shfl_sync(0xffffffffu, off, o + (uint32_t)st);
            if (t <= v) o += (uint32_t)st;
        }
        const uint32_t ooff = __shfl_sync(0xffffffffu, off, o);
        const uint32_t oqn = __shfl_sync(0xffffffffu, (uint32_t)qn, o);
        const uint32_t opix = __shfl_sync(0xffffffffu, ic.pix, o);
        PhiloxPrefix fo;
        fo.x0 = __shfl_sync(0xffffffffu, pf.x0, o);
        fo.n3 = __shfl_sync(0xffffffffu, pf.n3, o);
        fo.m1 = __shfl_sync(0xffffffffu, pf.m1, o);
        fo.hp0 = __shfl_sync(0xffffffffu, pf.hp0, o);
        fo.o3 = __shfl_sync(0xffffffffu, pf.o3, o);
        const bool valid = v < total;
        float c[B];
#pragma unroll
        for (int b = 0; b < B; ++b) c[b] = 0.0f;
        if (valid) {
            const uint32_t r = v - ooff;
            const uint32_t *oq = queue + wbase + o;
            uint32_t e = 0;                              // the owner's last entry with prefix <= r
#pragma unroll
            for (uint32_t st = 8; st > 0; st >>= 1)
                if (e + st < oqn && ((oq[(e + st) * bd] >> 8) & 0xFFu) <= r) e += st;
            const uint32_t m = oq[e * bd];
            uint32_t hm = m >> 16;
            for (uint32_t rr = r - ((m >> 8) & 0xFFu); rr; --rr) hm &= hm - 1u;
            const uint32_t bit = (uint32_t)(__ffs(hm) - 1);
            const uint32_t k = bit & 3u, q = bit >> 2, j = 4u * k + q;
            const uint8_t *rp = cb + (m & 0xFFu) * rec;
            const uint32_t gid = *reinterpret_cast<const uint32_t *>(rp);
            const uint4 w = philox_from_prefix_rk(fo, gid, a.rk0, a.rk1);
            const uint32_t hi = (word_of(w, k) >> (8u * q)) & 0xFFu;
            const uint32_t zc0 = rp[kRecZ7 + j] | rp[kRecZh + j];
            const uint32_t zc1 = rp[kRecZc1 + j];
            const uint32_t i = gid * (uint32_t)kGroup + j;
            uint32_t n;
            if (hi > zc0 && hi < zc1) {
                n = 1u;
            } else {
                const uint4 wlo = philox_rk(opix, i >> 2, ic.set, rng_tag(kKindLo, H, 0), a.rk0, a.rk1);
                const uint32_t x = (hi << 24) | (word_of(wlo, q) >> 8);
                const uint4 sr = __ldg(reinterpret_cast<const uint4 *>(ic.slow[H]) + i);
                n = count_from_thresholds(x, sr, ic.tail);
            }
            if (MODE == kModeCounts && n) {
                if (opix >= a.count_pix0 && opix - a.count_pix0 < a.count_npix)
                    a.counts[((size_t)(opix - a.count_pix0) * 2u + H) * a.n_points + i] = n;
            }
            if (n) {
                const float *f = ic.flux + (size_t)i * B;
                const float nf = (float)n;
#pragma unroll
                for (int b = 0; b < B; ++b) c[b] = __fmul_rn(nf, __ldg(f + b));
            }
        }
        // segmented inclusive scan over the list positions of one owner (owners ascend with v)
        const uint32_t key = valid ? o : 32u + lane;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t tk = __shfl_up_sync(0xffffffffu, key, d);
            float t[B];
#pragma unroll
            for (int b = 0; b < B; ++b) t[b] = __shfl_up_sync(0xffffffffu, c[b], d);
            if (lane >= (uint32_t)d && tk == key) {
#pragma unroll
                for (int b = 0; b < B; ++b) c[b] = __fadd_rn(c[b], t[b]);
            }
        }
        // this lane's segment in this pass ends at list position min(off + nb, v0 + 32) - 1
        const uint32_t s0 = max(off, v0), s1 = min(off + nb, v0 + 32u);
        const bool mine = s0 < s1;
        const uint32_t src = mine ? s1 - 1u - v0 : lane;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const float t = __shfl_sync(0xffffffffu, c[b], src);
            if (mine) part[b] = __fadd_rn(part[b], t);
        }
    }
    if (nb) acc.template add_sum<H>(part);
    __syncwarp();
}

// One staged chunk of groups: the HI call of every (pixel, group) from the pixel's Philox
// prefix, four byte-wise compares folded into a 16-bit maybe-hit mask, and one queue entry per
// group with maybe-hits (a predicated store, no per-bit loop); the warp drains the queues when
// one would overflow and at the chunk's end.
template <int B, bool KAHAN, int MODE, int H>
__device__ __forceinline__ void process_chunk(const DrawArgs &a, const ItemCtx &ic,
                                              const PhiloxPrefix &pf, const uint8_t *cb,
                                              uint32_t cnt, int sidx, uint32_t *queue,
                                              Acc<B, KAHAN> &acc) {
    constexpr uint32_t rec = kSparseRecBytes;
    uint32_t *myq = queue + threadIdx.x;
    const uint32_t bd = blockDim.x;
    // a lane queues at most one entry per group: with no more groups per lane than queue slots
    // in this chunk the queue cannot fill before the chunk's end
    const bool may_fill = (cnt + (uint32_t)a.split - 1u) / (uint32_t)a.split > (uint32_t)kQueueCap;
    int qn = 0;
#pragma unroll 2
    for (uint32_t g = (uint32_t)sidx; g < cnt; g += (uint32_t)a.split) {
        const uint8_t *r = cb + g * rec;
        const uint32_t gid = *reinterpret_cast<const uint32_t *>(r);
        const uint4 z7 = *reinterpret_cast<const uint4 *>(r + kRecZ7);
        const uint4 zh = *reinterpret_cast<const uint4 *>(r + kRecZh);
        const uint4 w = philox_from_prefix_rk(pf, gid, a.rk0, a.rk1);
        const uint32_t m0 = ge_bytes(w.x, z7.x, zh.x), m1 = ge_bytes(w.y, z7.y, zh.y);
        const uint32_t m2 = ge_bytes(w.z, z7.z, zh.z), m3 = ge_bytes(w.w, z7.w, zh.w);
        // maybe-hits of the 16 points: bit 8q + k of t is byte q of word k (point 4k + q), packed
        // into 16 bits as bit 4q + k
        uint32_t hm = ((m0 & 0x80808080u) >> 7) | ((m1 & 0x80808080u) >> 6) |
                      ((m2 & 0x80808080u) >> 5) | ((m3 & 0x80808080u) >> 4);
        hm = (hm | (hm >> 4)) & 0x00FF00FFu;
        hm = (hm | (hm >> 8)) & 0x0000FFFFu;
        // branch-free push: the entry goes to slot qn (< kQueueCap: a full queue is drained right
        // after the push that fills it) and counts only when it has maybe-hits
        myq[(uint32_t)qn * bd] = g | (hm << 16);
        qn += hm != 0u ? 1 : 0;
        if (may_fill && __any_sync(0xffffffffu, qn == kQueueCap)) {
            drain_warp<B, KAHAN, MODE, H>(a, ic, pf, cb, queue, qn, acc);
            qn = 0;
        }
    }
    if (__any_sync(0xffffffffu, qn > 0)) drain_warp<B, KAHAN, MODE, H>(a, ic, pf, cb, queue, qn, acc);
}

// One dense group (see process_dense), quad by quad: each quad's table entries are loaded at the
// quad's start.  The fused batched instantiation uses this form (the prefetching form below made
// its larger kernel slower).  WIDE: the word-table entries of a group with a mean of kWideLam or
// more (8-bit counts, bits 1-23 of the threshold, multi flag in bit 31); otherwise 7-bit counts,
// the multi flag in bit 7 and the low 24 bits of the threshold.
template <int B, bool KAHAN, int MODE, int H, bool WIDE>
__device__ __forceinline__ void dense_group_direct(const DrawArgs &a, const ItemCtx &ic, const uint8_t *r,
                                            uint32_t gid, const uint32_t *bt, const uint32_t *zg,
                                            const PhiloxPrefix &ph, const PhiloxPrefix &pl, Acc<B, KAHAN> &acc) {
    const uint4 whi = philox_from_prefix_rk(ph, gid, a.rk0, a.rk1);
    const float *fl = reinterpret_cast<const float *>(r + kRecFlux);
    const uint16_t *n0r = reinterpret_cast<const uint16_t *>(r + kRecN0);
    // the group's 16 contributions n f_b are summed with plain FMAs (at most 16 terms) and the
    // group total goes into the pixel's (compensated) accumulator once
    float gs[B];
#pragma unroll
    for (int b = 0; b < B; ++b) gs[b] = 0.0f;
#pragma unroll 2
    for (uint32_t qd = 0; qd < 4u; ++qd) {
        // the quad's four table entries and its 4 x B fluxes first: their loads overlap the LO call
        // (B 16-byte flux loads: the record's flux block is 16-byte aligned; with four bands each
        // slot's own 16-byte load below, fewer live registers)
        uint32_t e[4];
#pragma unroll
        for (uint32_t t = 0; t < 4u; ++t) {
            const uint32_t j = 4u * qd + t;
            e[t] = __ldg(bt + j * 256u + hi_byte(whi, j));
        }
        constexpr int kFq = B < 4 ? 4 * B : 1;
        float fq[kFq];
#pragma unroll
        for (int v = 0; v < (B < 4 ? B : 0); ++v) {
            const float4 f4 = __ldg(reinterpret_cast<const float4 *>(fl) + qd * (uint32_t)B + (uint32_t)v);
            fq[4 * v] = f4.x;
            fq[4 * v + 1] = f4.y;
            fq[4 * v + 2] = f4.z;
            fq[4 * v + 3] = f4.w;
        }
        const uint4 wlo = philox_from_prefix_rk(pl, gid * 4u + qd, a.rk0, a.rk1);
        const uint2 n0q = __ldg(reinterpret_cast<const uint2 *>(n0r) + qd);   // n0 of the quad's slots
#pragma unroll
        for (uint32_t t = 0; t < 4u; ++t) {
            const uint32_t j = 4u * qd + t;
            const uint32_t low = word_of(wlo, t) >> 8;
            uint32_t k;                                         // relative to n0
            if (WIDE) {
                const uint32_t l23 = low >> 1, z23 = (e[t] >> 8) & 0x7FFFFFu;
                k = e[t] & 0xFFu;
                if (!(e[t] & 0x80000000u) && l23 != z23) {
                    k += l23 > z23 ? 1u : 0u;
                } else {
                    // bits 1-23 equal (compare with the threshold itself), or several thresholds in
                    // the byte (walk from the stored count)
                    const uint32_t x = (hi_byte(whi, j) << 24) | low;
                    const uint32_t *zs = zg + j * (uint32_t)kTailCap;
                    const bool above = l23 != z23 ? l23 > z23 : x > __ldg(zs + k);
                    if (e[t] & 0x80000000u) k = above ? slot_up(x, zs, k + 1u) : slot_down(x, zs, k);
                    else k += above ? 1u : 0u;
                }
            } else {
                const bool above = low > (e[t] >> 8);
                k = (e[t] & 0x7Fu) + (above ? 1u : 0u);
                if (e[t] & 0x80u) {   // several thresholds in the byte: walk from the stored count
                    const uint32_t x = (hi_byte(whi, j) << 24) | low;
                    const uint32_t *zs = zg + j * (uint32_t)kTailCap;
                    k = above ? slot_up(x, zs, k) : slot_down(x, zs, k);
                }
            }
            const uint32_t n0s = ((t < 2u ? n0q.x : n0q.y) >> (16u * (t & 1u))) & 0xFFFFu;
            const uint32_t n = n0s + k;
            const float nf = (float)n;
            if (B < 4) {
#pragma unroll
                for (int b = 0; b < B; ++b) gs[b] = fmaf(nf, fq[(t * B + b) % kFq], gs[b]);
            } else {
                const float4 f4 = __ldg(reinterpret_cast<const float4 *>(fl) + j);
                const float fs[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
                for (int b = 0; b < B; ++b) gs[b] = fmaf(nf, fs[b % 4], gs[b]);
            }
            if (MODE == kModeCounts && n) {
                if (ic.pix >= a.count_pix0 && ic.pix - a.count_pix0 < a.count_npix)
                    a.counts[((size_t)(ic.pix - a.count_pix0) * 2u + H) * a.n_points + gid * (uint32_t)kGroup + j] = n;
            }
        }
    }
    acc.template add_sum<H>(gs);
}

// One dense group (see process_dense), with its table entries loaded two quads ahead of their use
// and, for a narrow group's bytes with several thresholds, the two thresholds bounding the stored
// count loaded before the LO call (a word of that count then needs no further load).  Used by the
// image and counts instantiations.
template <int B, bool KAHAN, int MODE, int H, bool WIDE>
__device__ __forceinline__ void dense_group(const DrawArgs &a, const ItemCtx &ic, const uint8_t *r,
                                            uint32_t gid, const uint32_t *bt, const uint32_t *zg,
                                            const PhiloxPrefix &ph, const PhiloxPrefix &pl, Acc<B, KAHAN> &acc) {
    const uint4 whi = philox_from_prefix_rk(ph, gid, a.rk0, a.rk1);
    const float *fl = reinterpret_cast<const float *>(r + kRecFlux);
    const uint16_t *n0r = reinterpret_cast<const uint16_t *>(r + kRecN0);
    constexpr uint32_t kMulti = WIDE ? 0x80000000u : 0x80u, kCount = WIDE ? 0xFFu : 0x7Fu;
    // the table entries of a quad (issued two quads ahead of their use)
    uint32_t ring[4][4];
    auto load_quad = [&](uint32_t qd, uint32_t (&e)[4]) {
#pragma unroll
        for (uint32_t t = 0; t < 4u; ++t) {
            const uint32_t j = 4u * qd + t;
            e[t] = __ldg(bt + j * 256u + hi_byte(whi, j));
        }
    };
    load_quad(0u, ring[0]);
    load_quad(1u, ring[1]);
    // the group's 16 contributions n f_b are summed with plain FMAs (at most 16 terms) and the
    // group total goes into the pixel's (compensated) accumulator once
    float gs[B];
#pragma unroll
    for (int b = 0; b < B; ++b) gs[b] = 0.0f;
#pragma unroll
    for (uint32_t qd = 0; qd < 4u; ++qd) {
        if (qd < 2u) load_quad(qd + 2u, ring[qd + 2u]);
        // narrow layout, a byte with several thresholds: its count's two bounding thresholds
        // Z_(n0+c-1), Z_(n0+c) are loaded before the LO call, so that a word of count c needs no
        // further load (wide groups, where such bytes are frequent, load only on a walk)
        uint32_t zb[4], zt[4];
#pragma unroll
        for (uint32_t t = 0; t < 4u; ++t) {
            const uint32_t e = ring[qd][t];
            zb[t] = 0u;
            zt[t] = 0u;
            if (!WIDE && (e & kMulti)) {
                const uint32_t *zs = zg + (4u * qd + t) * (uint32_t)kTailCap;
                const uint32_t k = e & kCount;
                zt[t] = __ldg(zs + k);
                if (k) zb[t] = __ldg(zs + k - 1u);
            }
        }
        // the quad's 4 x B fluxes: B 16-byte loads (the record's flux block is 16-byte aligned);
        // with four bands each slot's own 16-byte load below (fewer live registers)
        constexpr int kFq = B < 4 ? 4 * B : 1;
        float fq[kFq];
#pragma unroll
        for (int v = 0; v < (B < 4 ? B : 0); ++v) {
            const float4 f4 = __ldg(reinterpret_cast<const float4 *>(fl) + qd * (uint32_t)B + (uint32_t)v);
            fq[4 * v] = f4.x;
            fq[4 * v + 1] = f4.y;
            fq[4 * v + 2] = f4.z;
            fq[4 * v + 3] = f4.w;
        }
        const uint4 wlo = philox_from_prefix_rk(pl, gid * 4u + qd, a.rk0, a.rk1);
        const uint2 n0q = __ldg(reinterpret_cast<const uint2 *>(n0r) + qd);   // n0 of the quad's slots
#pragma unroll
        for (uint32_t t = 0; t < 4u; ++t) {
            const uint32_t j = 4u * qd + t;
            const uint32_t e = ring[qd][t];
            const uint32_t low = word_of(wlo, t) >> 8;
            uint32_t k = e & kCount;                            // relative to n0
            if (e & kMulti) {
                // several thresholds in the byte: count k for Z_(k-1) < x <= Z_k, else a walk
                const uint32_t x = (hi_byte(whi, j) << 24) | low;
                const uint32_t *zs = zg + j * (uint32_t)kTailCap;
                if (WIDE) {
                    const uint32_t l23 = low >> 1, z23 = (e >> 8) & 0x7FFFFFu;
                    const bool above = l23 != z23 ? l23 > z23 : x > __ldg(zs + k);
                    k = above ? slot_up(x, zs, k + 1u) : slot_down(x, zs, k);
                } else if (x > zt[t]) {
                    k = slot_up(x, zs, k + 1u);
                } else if (k && x <= zb[t]) {
                    k = slot_down(x, zs, k - 1u);
                }
            } else if (WIDE) {
                const uint32_t l23 = low >> 1, z23 = (e >> 8) & 0x7FFFFFu;
                if (l23 != z23) {
                    k += l23 > z23 ? 1u : 0u;
                } else {   // bits 1-23 equal: compare with the threshold itself
                    const uint32_t x = (hi_byte(whi, j) << 24) | low;
                    k += x > __ldg(zg + j * (uint32_t)kTailCap + k) ? 1u : 0u;
                }
            } else {
                k += low > (e >> 8) ? 1u : 0u;
            }
            const uint32_t n0s = ((t < 2u ? n0q.x : n0q.y) >> (16u * (t & 1u))) & 0xFFFFu;
            const uint32_t n = n0s + k;
            const float nf = (float)n;
            if (B < 4) {
#pragma unroll
                for (int b = 0; b < B; ++b) gs[b] = fmaf(nf, fq[(t * B + b) % kFq], gs[b]);
            } else {
                const float4 f4 = __ldg(reinterpret_cast<const float4 *>(fl) + j);
                const float fs[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
                for (int b = 0; b < B; ++b) gs[b] = fmaf(nf, fs[b % 4], gs[b]);
            }
            if (MODE == kModeCounts && n) {
                if (ic.pix >= a.count_pix0 && ic.pix - a.count_pix0 < a.count_npix)
                    a.counts[((size_t)(ic.pix - a.count_pix0) * 2u + H) * a.n_points + gid * (uint32_t)kGroup + j] = n;
            }
        }
    }
    acc.template add_sum<H>(gs);
}

// Dense inversion groups (a slot with lambda >= kDenseLam): nearly every slot is non-zero, so
// the HI call and the four LO calls of the group are drawn up front.  Each slot's count comes
// from its word table and the slot's leading count n0 (kept in the group record): n0 plus the
// table's count at the lower edge of the HI byte, plus one when the word is above the byte's
// first threshold (decided from the threshold bits stored in the entry).  A byte holding two or
// more thresholds (the tails of the distribution) starts at its most frequent count m instead
// and walks through the point's threshold slot from there, upwards when the word is above Z_m,
// downwards otherwise.  A group's entry format (record header word 1) is the same for all its
// lanes, so the branch on it does not diverge.
template <int B, bool KAHAN, int MODE, int H>
__device__ __forceinline__ void process_dense(const DrawArgs &a, const ItemCtx &ic, const SetDesc &d,
                                              int sidx, Acc<B, KAHAN> &acc) {
    constexpr uint32_t rec = group_rec_bytes(B);
    const uint32_t nd = ic.active ? d.n_dense[H] : 0u;
    if (nd == 0u) return;
    const uint8_t *base = a.tables + d.dense_off[H];
    const uint32_t *btab = reinterpret_cast<const uint32_t *>(a.btab + d.btab_off[H]);
    // threshold slots of this half: kTailCap words per point slot, 16 G point slots per half
    const uint32_t *zh = ic.tail + (size_t)H * ((a.n_points + kGroup - 1u) / kGroup) * kGroup * kTailCap;
    const PhiloxPrefix ph = philox_prefix_rk(ic.pix, ic.set, rng_tag(kKindHi, H, 0), a.rk0, a.rk1);
    const PhiloxPrefix pl = philox_prefix_rk(ic.pix, ic.set, rng_tag(kKindLo, H, 0), a.rk0, a.rk1);
    for (uint32_t q = (uint32_t)sidx; q < nd; q += (uint32_t)a.split) {
        const uint8_t *r = base + (size_t)q * rec;
        const uint2 hd = __ldg(reinterpret_cast<const uint2 *>(r));     // group id, wide format
        const uint32_t *bt = btab + (size_t)q * kBtabGroupEntries;
        const uint32_t *zg = zh + (size_t)hd.x * kGroup * kTailCap;
        if (MODE == kModeFused) {
            if (hd.y) dense_group_direct<B, KAHAN, MODE, H, true>(a, ic, r, hd.x, bt, zg, ph, pl, acc);
            else dense_group_direct<B, KAHAN, MODE, H, false>(a, ic, r, hd.x, bt, zg, ph, pl, acc);
        } else {
            if (hd.y) dense_group<B, KAHAN, MODE, H, true>(a, ic, r, hd.x, bt, zg, ph, pl, acc);
            else dense_group<B, KAHAN, MODE, H, false>(a, ic, r, hd.x, bt, zg, ph, pl, acc);
        }
    }
}

__device__ __forceinline__ PtrsRec load_ptrs(const PtrsRec *pr, uint32_t q) {
    PtrsRec rec;
    const uint4 *src = reinterpret_cast<const uint4 *>(pr + q);
    uint4 *dst = reinterpret_cast<uint4 *>(&rec);
    dst[0] = __ldg(src);
    dst[1] = __ldg(src + 1);
    dst[2] = __ldg(src + 2);
    return rec;
}

template <int B, bool KAHAN, int MODE, int H>
__device__ __forceinline__ void ptrs_resolved(const DrawArgs &a, const ItemCtx &ic, const PtrsRec &rec,
                                              uint32_t n, Acc<B, KAHAN> &acc) {
    if (!n) return;
    acc.template add<H>((float)n, rec.flux);
    if (MODE == kModeCounts) {
        if (ic.pix >= a.count_pix0 && ic.pix - a.count_pix0 < a.count_npix)
            a.counts[((size_t)(ic.pix - a.count_pix0) * 2u + H) * a.n_points + rec.i] = n;
    }
}


// Total-count sampler of half H (the Section 2.1 footnote's additivity of Poisson counts, used
// in reverse: a Poisson total split over the points by their weights gives independent Poisson
// counts): N ~ Poisson(Lambda) from word 0 of Philox(p, 2^32 - 1, set, LO|H)
// by inversion (Lambda < 10) or by transformed rejection with point index 2^32 - 1; star s takes
// word s & 3 of Philox(p, 2^31 | s >> 2, set, HI|H) and goes to the first pool entry with
// u < T_j (the last takes the rest): the top 14 bits of u select a guide bucket, a binary
// search inside it finds the entry (bounded, so no lane walks a long run of tiny weights).
template <int B, bool KAHAN, int MODE, int H>
__device__ __forceinline__ void process_pool(const DrawArgs &a, const ItemCtx &ic, const SetDesc &d,
                                             int sidx, Acc<B, KAHAN> &acc) {
    if (!ic.active || sidx != H % a.split) return;
    const uint8_t *pr = a.tables + d.pool_off[H];
    const PoolHdr hdr = *reinterpret_cast<const PoolHdr *>(pr);
    const uint32_t mode = hdr.mode & 0xFFu;
    if (mode == 0u || hdr.n == 0u) return;
    uint32_t n_star;
    if (mode == 1u) {
        // n0 leading thresholds of -1 (bits 8-15 of the mode word), then the walk
        const uint32_t x = philox_rk(ic.pix, 0xFFFFFFFFu, ic.set, rng_tag(kKindLo, H, 0), a.rk0, a.rk1).x;
        const uint32_t *z = reinterpret_cast<const uint32_t *>(pr + kPoolZOff);
        uint32_t k = 0u;
        while (k < hdr.n_z && x > __ldg(z + k)) ++k;
        n_star = ((hdr.mode >> 8) & 0xFFu) + k;
    } else {
        const PtrsRec rec = load_ptrs(reinterpret_cast<const PtrsRec *>(pr + kPoolPtrsOff), 0u);
        n_star = ptrs_draw(rec, ic.pix, ic.set, H, a.rk0, a.rk1, a.ptrs_cap, a.err);
    }
    const uint32_t *guide = reinterpret_cast<const uint32_t *>(pr + kPoolGuideOff);
    const uint32_t *idx = reinterpret_cast<const uint32_t *>(pr + kPoolIdxOff);
    const uint32_t *thr = idx + hdr.n;
    const float *flux = reinterpret_cast<const float *>(a.tables + d.flux_off);
    uint4 w = make_uint4(0, 0, 0, 0);
    for (uint32_t st = 0; st < n_star; ++st) {
        if ((st & 3u) == 0u)
            w = philox_rk(ic.pix, 0x80000000u | (st >> 2), ic.set, rng_tag(kKindHi, H, 0), a.rk0, a.rk1);
        const uint32_t u = word_of(w, st & 3u);
        // the entry lies in [guide[b], guide[b + 1]]: binary search for the first j with
        // u < T_j (the last entry takes every remaining u)
        const uint32_t b = u >> (32 - kPoolGuideBits);
        uint32_t lo = __ldg(guide + b), hi = __ldg(guide + b + 1);
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (u < __ldg(thr + mid)) hi = mid;
            else lo = mid + 1u;
        }
        const uint32_t i = __ldg(idx + lo);
        float f[B];
#pragma unroll
        for (int b = 0; b < B; ++b) f[b] = __ldg(flux + (size_t)i * B + b);
        acc.template add<H>(1.0f, f);
        if (MODE == kModeCounts) {
            if (ic.pix >= a.count_pix0 && ic.pix - a.count_pix0 < a.count_npix)
                a.counts[((size_t)(ic.pix - a.count_pix0) * 2u + H) * a.n_points + i] += 1u;
        }
    }
}

// Transformed-rejection points (lambda >= 640) of half H.  The lanes (pixels) of a warp start on
// the records q = sidx, sidx + split, ... and every iteration of a warp-wide loop makes one
// cheap attempt for each lane's current draw: a squeeze acceptance gives the count and moves
// the lane to its next record, a quick rejection moves it to the draw's next attempt, and an
// attempt the squeeze leaves open waits for the log-form test.  The waiting lanes take their
// log-form tests together, once kPtrsLogBatch of them wait or every live lane does, so the
// warp runs the expensive test a few times per draw round instead of in nearly every
// iteration.  Each draw still takes exactly the attempt loop's decisions in order (first
// accepted attempt, cap as in ptrs_draw): a waiting lane makes no further attempt of its draw
// until its test is decided.  Called by all 32 lanes of the warp.
constexpr int kPtrsLogBatch = 16;

template <int B, bool KAHAN, int MODE, int H>
__device__ __forceinline__ void process_ptrs(const DrawArgs &a, const ItemCtx &ic, const SetDesc &d,
                                             int sidx, Acc<B, KAHAN> &acc) {
    const uint32_t n_rec = d.n_ptrs[H];
    if (n_rec == 0u) return;
    const PtrsRec *pr = reinterpret_cast<const PtrsRec *>(a.tables + d.ptrs_off[H]);
    uint32_t q = ic.active ? (uint32_t)sidx : n_rec;
    uint32_t at = 0;
    PtrsRec rec;
    if (q < n_rec) rec = load_ptrs(pr, q);
    uint4 w = make_uint4(0, 0, 0, 0);
    PtrsTry t;
    t.kf = t.us = t.V = 0.0f;
    t.status = 1;
    bool wait = false;          // the current attempt waits for its log-form test
    // accepted draws' n f_b are summed with plain FMAs, 32 draws at a time, and each partial goes
    // into the pixel's (compensated) accumulator
    float ps[B];
#pragma unroll
    for (int b = 0; b < B; ++b) ps[b] = 0.0f;
    uint32_t np = 0u;
    // the draw of record q ends: accepted with count n, or (ok false) the attempt cap was reached
    auto finish = [&](uint32_t n, bool ok) {
        if (ok) {
            const float nf = (float)n;
#pragma unroll
            for (int b = 0; b < B; ++b) ps[b] = fmaf(nf, rec.flux[b], ps[b]);
            if (++np == 32u) {
                acc.template add_sum<H>(ps);
#pragma unroll
                for (int b = 0; b < B; ++b) ps[b] = 0.0f;
                np = 0u;
            }
            if (MODE == kModeCounts && n) {
                if (ic.pix >= a.count_pix0 && ic.pix - a.count_pix0 < a.count_npix)
                    a.counts[((size_t)(ic.pix - a.count_pix0) * 2u + H) * a.n_points + rec.i] = n;
            }
        } else {
            atomicOr(a.err, kErrSampler);
        }
        q += (uint32_t)a.split;
        at = 0u;
        if (q < n_rec) rec = load_ptrs(pr, q);
    };
    for (;;) {
        const uint32_t live = __ballot_sync(0xffffffffu, q < n_rec);
        if (live == 0u) break;
        const uint32_t waiting = __ballot_sync(0xffffffffu, wait);
        if (waiting != 0u && (__popc(waiting) >= kPtrsLogBatch || waiting == live) && wait) {
            wait = false;
            if (ptrs_log_accept(rec, t)) finish((uint32_t)t.kf, true);
            else if (++at >= a.ptrs_cap) finish(0u, false);
        }
        if (q < n_rec && !wait) {
            if ((at & 1u) == 0u) w = ptrs_words(rec, ic.pix, ic.set, H, at, a.rk0, a.rk1);
            t = ptrs_cheap(rec, (at & 1u) ? w.z : w.x, (at & 1u) ? w.w : w.y);
            if (t.status == 0) finish((uint32_t)t.kf, true);
            else if (t.status == 2) wait = true;
            else if (++at >= a.ptrs_cap) finish(0u, false);
        }
    }
    if (np) acc.template add_sum<H>(ps);
}

// Dust screen factors of one pixel: E(B-V) = 10^log_ebv exp(sigma z), z ~ N(0, 1) by
// Box-Muller from Philox(p, 0, set, DUST); factor_b = 10^(-0.4 R_b E).
template <int B>
__device__ __forceinline__ void dust_factors(const SetDesc &d, uint32_t pix, uint32_t k0,
                                             uint32_t k1, float (&fac)[B]) {
    float z = 0.0f;
    if (d.dust_sigma != 0.0f) {
        const uint4 w = philox(pix, 0u, d.set_id, rng_tag(kKindDust, 0, 0), k0, k1);
        const float u1 = uniform_of(w.x), u2 = uniform_of(w.y);
        z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    }
    const float e = expf(d.dust_a + d.dust_sigma * z);
#pragma unroll
    for (int b = 0; b < B; ++b) fac[b] = exp10f(d.dust_c[b] * e);
}

// PATHS: which draw paths are compiled in besides the sparse inversion groups: kPathDense (dense
// groups and transformed-rejection points), kPathPool (the total-count sampler in place of the
// inversion groups), or both.  The host picks the smallest set its models can need.
template <int B, bool KAHAN, int MODE, int PATHS>
__global__ void __launch_bounds__(256, (PATHS & kPathDense) ? 2 : ((PATHS & kPathPool) ? 4 : 3)) draw_kernel(const __grid_constant__ DrawArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr uint32_t rec = kSparseRecBytes;   // staged sparse group records
    const uint32_t chunk = (uint32_t)a.chunk;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    volatile uint32_t *s_item = reinterpret_cast<volatile uint32_t *>(smem + 16);
    uint32_t *s_ntouch = reinterpret_cast<uint32_t *>(smem + 20);
    uint8_t *bufs = smem + 32;
    uint32_t *queue = reinterpret_cast<uint32_t *>(bufs + chunk_region_bytes(chunk, rec));
    float *red = reinterpret_cast<float *>(queue + (size_t)kQueueCap * blockDim.x);
    const int tid = threadIdx.x;
    const int ppc = blockDim.x / a.split;
    const int sidx = tid / ppc;
    const int pl = tid - sidx * ppc;
    uint32_t *hist = reinterpret_cast<uint32_t *>(red + (size_t)blockDim.x * 2 * B);
    const int nbins = a.pc.nx * a.pc.ny;
    uint32_t *touched = hist + nbins;
    double *wred = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(touched + ppc) + 7u) & ~uintptr_t(7));
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        *s_ntouch = 0u;
    }
    if (MODE == kModeFused)
        for (int i = tid; i < nbins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    uint32_t parity = 0u;
    uint32_t pending = 0u;   // bit b: buffer b has an issued, not yet awaited copy

    for (uint32_t q = blockIdx.x;; q += gridDim.x) {
        uint32_t pos;
        if (a.queue) {
            if (tid == 0) *s_item = atomicAdd(a.queue, 1u);
            __syncthreads();
            pos = *s_item;
        } else {
            pos = q;
        }
        if (pos >= a.n_items) break;
        const uint32_t item = a.order ? __ldg(a.order + pos) : pos;
        const uint2 it = a.items[item];
        const SetDesc &d = a.desc[it.x];
        ItemCtx ic;
        ic.npix = d.n_im * d.n_im;
        ic.pix = it.y * (uint32_t)ppc + (uint32_t)pl;
        ic.active = ic.pix < ic.npix;
        ic.set = d.set_id;
        ic.slow[0] = reinterpret_cast<const SlowRec *>(a.tables + d.slow_off[0]);
        ic.slow[1] = reinterpret_cast<const SlowRec *>(a.tables + d.slow_off[1]);
        ic.tail = reinterpret_cast<const uint32_t *>(a.tables + d.tail_off);
        ic.flux = reinterpret_cast<const float *>(a.tables + d.flux_off);
        Acc<B, KAHAN> acc;
        acc.init();

        // ---- inversion points, streamed through shared memory chunk by chunk (or, with the
        // total-count sampler, drawn through the pool) ----
        const uint32_t ng0 = d.pool_on ? 0u : d.n_grp[0], ng1 = d.pool_on ? 0u : d.n_grp[1];
        const uint32_t nc0 = (ng0 + chunk - 1) / chunk, nc1 = (ng1 + chunk - 1) / chunk;
        const uint32_t nc = nc0 + nc1;
        // Chunk c + 1 is copied while chunk c is processed.  Every thread waits for a chunk's
        // copy at the end of the previous chunk (or before the first); the barrier after the
        // wait tells the whole CTA whether any wait ran out, in which case the copy stays
        // pending (the final drain waits for it), no chunk is read from an unfilled buffer and
        // the CTA stops (the error is latched).
        bool stop = false;
        if (tid == 0 && nc > 0) {
            const uint32_t cnt = min(chunk, nc0 > 0 ? ng0 : ng1);
            const uint8_t *src = a.tables + (nc0 > 0 ? d.grp_off[0] : d.grp_off[1]);
            mbar_expect_tx(&bars[0], cnt * rec);
            bulk_g2s(bufs, src, cnt * rec, &bars[0]);
            pending |= 1u;
        }
        if (nc > 0) {
            const bool ok = mbar_wait(&bars[0], parity & 1u, a.err) || mbar_wait(&bars[0], parity & 1u, a.err);
            stop = __syncthreads_or(!ok) != 0;
            if (!stop) {
                parity ^= 1u;
                pending &= ~1u;
            }
        }
        for (uint32_t c = 0; c < nc && !stop; ++c) {
            const uint32_t b = c & 1u, bn = b ^ 1u;
            if (tid == 0 && c + 1 < nc) {
                const uint32_t cn = c + 1;
                const uint32_t h = cn >= nc0 ? 1u : 0u;
                const uint32_t first = (h ? cn - nc0 : cn) * chunk;
                const uint32_t cnt = min(chunk, (h ? ng1 : ng0) - first);
                mbar_expect_tx(&bars[bn], cnt * rec);
                bulk_g2s(bufs + bn * chunk * rec, a.tables + d.grp_off[h] + (uint64_t)first * rec,
                         cnt * rec, &bars[bn]);
                pending |= 1u << bn;
            }
            const uint32_t h = c >= nc0 ? 1u : 0u;
            const uint32_t first = (h ? c - nc0 : c) * chunk;
            const uint32_t cnt = min(chunk, (h ? ng1 : ng0) - first);
            const uint8_t *cb = bufs + b * chunk * rec;
            // the pixel's HI-call prefix of this half (rounds 1-3 without the group index)
            const PhiloxPrefix pf = philox_prefix_rk(ic.pix, ic.set, rng_tag(kKindHi, h, 0), a.rk0, a.rk1);
            if (h == 0u) process_chunk<B, KAHAN, MODE, 0>(a, ic, pf, cb, cnt, sidx, queue, acc);
            else process_chunk<B, KAHAN, MODE, 1>(a, ic, pf, cb, cnt, sidx, queue, acc);
            bool ok = true;
            if (c + 1 < nc) {
                const uint32_t par = (parity >> bn) & 1u;
                ok = mbar_wait(&bars[bn], par, a.err) || mbar_wait(&bars[bn], par, a.err);
            }
            stop = __syncthreads_or(!ok) != 0;
            if (!stop && c + 1 < nc) {
                parity ^= 1u << bn;
                pending &= ~(1u << bn);
            }
        }
        if (stop) break;

        // ---- dense inversion groups, then transformed-rejection points (lambda >= 640) ----
        if (PATHS & kPathPool) {
            process_pool<B, KAHAN, MODE, 0>(a, ic, d, sidx, acc);
            process_pool<B, KAHAN, MODE, 1>(a, ic, d, sidx, acc);
        } else if (PATHS & kPathDense) {
            process_dense<B, KAHAN, MODE, 0>(a, ic, d, sidx, acc);
            process_dense<B, KAHAN, MODE, 1>(a, ic, d, sidx, acc);
        }
        if (PATHS & kPathDense) {
            process_ptrs<B, KAHAN, MODE, 0>(a, ic, d, sidx, acc);
            process_ptrs<B, KAHAN, MODE, 1>(a, ic, d, sidx, acc);
        }

        // ---- combine the splits of each pixel in a fixed order ----
        float v0[B], v1[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            v0[b] = acc.template value<0>(b);
            v1[b] = acc.template value<1>(b);
        }
        if (a.split > 1) {
            float *my = red + (size_t)tid * 2 * B;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                my[b] = v0[b];
                my[B + b] = v1[b];
            }
            __syncthreads();
            if (sidx == 0) {
                for (int s = 1; s < a.split; ++s) {
                    const float *o = red + (size_t)(s * ppc + pl) * 2 * B;
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        v0[b] = __fadd_rn(v0[b], o[b]);
                        v1[b] = __fadd_rn(v1[b], o[B + b]);
                    }
                }
            }
        }

        // ---- epilogue: dust screen, then image store or the fused pixel stage ----
        float F[B];
        const bool own = sidx == 0 && ic.active;
        if (own) {
            if (d.dust_on) {
                float fac[B];
                dust_factors<B>(d, ic.pix, k0, k1, fac);
#pragma unroll
                for (int b = 0; b < B; ++b) F[b] = v0[b] + fac[b] * v1[b];
            } else {
#pragma unroll
                for (int b = 0; b < B; ++b) F[b] = __fadd_rn(v0[b], v1[b]);
            }
        }
        if (MODE == kModeImage) {
            if (own) {
#pragma unroll
                for (int b = 0; b < B; ++b) a.image[d.img_off + (size_t)b * ic.npix + ic.pix] = F[b];
            }
        } else if (MODE == kModeFused) {
            double cs = 0.0, ms = 0.0, nv = 0.0;
            uint32_t novf = 0u, ninv = 0u;
            if (sidx == 0) {
                int bin = -1;
                if (ic.active) {
                    const PixelOut o = pixel_stage<B>(F, ic.pix, ic.set, a.pc);
                    if (o.valid) {
                        cs = (double)__fsub_rn(o.col, a.pc.c_lo);
                        ms = (double)__fsub_rn(o.mag, a.pc.m_lo);
                        nv = 1.0;
                        bin = o.bin;
                        if (bin < 0) novf = 1u;
                    } else {
                        ninv = 1u;
                    }
                }
                hist_add_warp(hist, touched, s_ntouch, bin, (uint32_t)ppc);
            }
            // block reduction of the item's moments and counters
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                cs += __shfl_xor_sync(0xffffffffu, cs, o);
                ms += __shfl_xor_sync(0xffffffffu, ms, o);
                nv += __shfl_xor_sync(0xffffffffu, nv, o);
                novf += __shfl_xor_sync(0xffffffffu, novf, o);
                ninv += __shfl_xor_sync(0xffffffffu, ninv, o);
            }
            const int wid = tid >> 5, lane = tid & 31;
            if (lane == 0) {
                wred[wid * 5 + 0] = cs;
                wred[wid * 5 + 1] = ms;
                wred[wid * 5 + 2] = nv;
                wred[wid * 5 + 3] = (double)novf;
                wred[wid * 5 + 4] = (double)ninv;
            }
            __syncthreads();
            const uint32_t nbins_u = (uint32_t)nbins;
            const uint32_t ntouch = min(*s_ntouch, (uint32_t)ppc);
            uint32_t *gh = a.hess + (size_t)it.x * nbins_u;
            for (uint32_t t = tid; t < ntouch; t += blockDim.x) {
                const uint32_t bin = touched[t];
                const uint32_t v = hist[bin];
                hist[bin] = 0u;
                if (v) atomicAdd(gh + bin, v);
            }
            if (tid == 0) {
                double t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    t0 += wred[w * 5 + 0];
                    t1 += wred[w * 5 + 1];
                    t2 += wred[w * 5 + 2];
                    t3 += wred[w * 5 + 3];
                    t4 += wred[w * 5 + 4];
                }
                a.item_moments[(size_t)item * 3 + 0] = t0 + t2 * (double)a.pc.c_lo;
                a.item_moments[(size_t)item * 3 + 1] = t1 + t2 * (double)a.pc.m_lo;
                a.item_moments[(size_t)item * 3 + 2] = t2;
                if (t3 > 0.0) atomicAdd(a.counters + (size_t)it.x * 2 + 0, (uint32_t)t3);
                if (t4 > 0.0) atomicAdd(a.counters + (size_t)it.x * 2 + 1, (uint32_t)t4);
            }
            __syncthreads();
            if (tid == 0) *s_ntouch = 0u;
        }
        __syncthreads();
        if (!a.queue) break;
    }
    // a copy can only be outstanding here after a timed-out wait: wait for it once more before
    // the CTA (and its shared memory) goes away
    if (tid == 0) {
        for (uint32_t b = 0; b < 2; ++b)
            if (pending & (1u << b)) mbar_wait(&bars[b], (parity >> b) & 1u, a.err);
    }
}

// ---- launch helpers, instantiated by the translation unit that owns each PATHS value ----
// Opt in to the dynamic shared memory of each instantiation once per process (before any
// stream capture: the first call of every configuration goes through the occupancy query).
template <int B, bool KAHAN, int MODE, int PATHS>
static cudaError_t configure_t(size_t smem) {
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(draw_kernel<B, KAHAN, MODE, PATHS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    return cudaSuccess;
}

template <int B, bool KAHAN, int MODE, int PATHS>
static cudaError_t launch_t(const DrawArgs &a, int grid, int block, size_t smem, cudaStream_t st) {
    cudaError_t e = configure_t<B, KAHAN, MODE, PATHS>(smem);
    if (e != cudaSuccess) return e;
    draw_kernel<B, KAHAN, MODE, PATHS><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int B, bool KAHAN, int MODE, int PATHS>
static int occupancy_t(int block, size_t smem) {
    if (configure_t<B, KAHAN, MODE, PATHS>(smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, draw_kernel<B, KAHAN, MODE, PATHS>, block, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

template <int B, bool KAHAN, int PATHS>
static int occupancy_m(int mode, int block, size_t smem) {
    switch (mode) {
        case kModeImage: return occupancy_t<B, KAHAN, kModeImage, PATHS>(block, smem);
        case kModeCounts: return occupancy_t<B, KAHAN, kModeCounts, PATHS>(block, smem);
        default: return occupancy_t<B, KAHAN, kModeFused, PATHS>(block, smem);
    }
}

template <int PATHS>
static int occupancy_paths(int nb, bool kahan, int mode, int block, size_t smem) {
    switch (nb) {
        case 2: return kahan ? occupancy_m<2, true, PATHS>(mode, block, smem) : occupancy_m<2, false, PATHS>(mode, block, smem);
        case 3: return kahan ? occupancy_m<3, true, PATHS>(mode, block, smem) : occupancy_m<3, false, PATHS>(mode, block, smem);
        default: return kahan ? occupancy_m<4, true, PATHS>(mode, block, smem) : occupancy_m<4, false, PATHS>(mode, block, smem);
    }
}

template <int B, bool KAHAN, int PATHS>
static cudaError_t launch_m(const DrawArgs &a, int mode, int grid, int block, size_t smem, cudaStream_t st) {
    switch (mode) {
        case kModeImage: return launch_t<B, KAHAN, kModeImage, PATHS>(a, grid, block, smem, st);
        case kModeCounts: return launch_t<B, KAHAN, kModeCounts, PATHS>(a, grid, block, smem, st);
        default: return launch_t<B, KAHAN, kModeFused, PATHS>(a, grid, block, smem, st);
    }
}

template <int PATHS>
static cudaError_t launch_paths(const DrawArgs &a, int nb, bool kahan, int mode, int grid, int block, size_t smem,
                                cudaStream_t st) {
    switch (nb) {
        case 2: return kahan ? launch_m<2, true, PATHS>(a, mode, grid, block, smem, st)
                             : launch_m<2, false, PATHS>(a, mode, grid, block, smem, st);
        case 3: return kahan ? launch_m<3, true, PATHS>(a, mode, grid, block, smem, st)
                             : launch_m<3, false, PATHS>(a, mode, grid, block, smem, st);
        default: return kahan ? launch_m<4, true, PATHS>(a, mode, grid, block, smem, st)
                              : launch_m<4, false, PATHS>(a, mode, grid, block, smem, st);
    }
}

}  // namespace pcmd
