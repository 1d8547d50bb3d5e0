// Device helpers of libpcmd: counter-based RNG, the sampler's FP32 arithmetic, bulk-copy
// staging with bounded mbarrier waits, and the per-pixel noise / magnitude / Hess-bin stage.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>
#include "pcmd_internal.h"

namespace pcmd {

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011): 10 rounds of two 32x32->64 multiplies
// with the Weyl key schedule.  Counter (pixel, index, set, tag), key = 64-bit seed.
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Philox of counters (c0, c1 = varying index, c2, c3) with c0, c2, c3 and the key fixed: the
// parts of rounds 1-3 that do not depend on c1 are computed once (PhiloxPrefix), leaving one
// XOR in round 1, one multiply in rounds 2 and 3 and seven full rounds per call.
struct PhiloxPrefix {
    uint32_t x0;        // round 1: hi(M1 c2) ^ k0                   (c1 enters by XOR)
    uint32_t n3;        // round 1: lo(M0 c0)
    uint32_t m0, m1;    // round 2 outputs 0 and 1 (independent of c1)
    uint32_t hp0, o3;   // round 3: hi and lo of M0 m0
    uint32_t k0, k1;
};

__host__ __device__ __forceinline__ PhiloxPrefix philox_prefix(uint32_t c0, uint32_t c2, uint32_t c3,
                                                             uint32_t k0, uint32_t k1) {
    PhiloxPrefix f;
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    f.x0 = (uint32_t)(p1 >> 32) ^ k0;
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    f.n3 = (uint32_t)p0;
    const uint64_t q1 = (uint64_t)0xCD9E8D57u * (uint64_t)n2;
    f.m0 = (uint32_t)(q1 >> 32) ^ n1 ^ (k0 + 0x9E3779B9u);
    f.m1 = (uint32_t)q1;
    const uint64_t r0 = (uint64_t)0xD2511F53u * (uint64_t)f.m0;
    f.hp0 = (uint32_t)(r0 >> 32);
    f.o3 = (uint32_t)r0;
    f.k0 = k0;
    f.k1 = k1;
    return f;
}

__host__ __device__ __forceinline__ uint4 philox_from_prefix(const PhiloxPrefix &f, uint32_t c1) {
    const uint32_t n0 = f.x0 ^ c1;
    const uint64_t q0 = (uint64_t)0xD2511F53u * (uint64_t)n0;
    const uint32_t m2 = (uint32_t)(q0 >> 32) ^ f.n3 ^ (f.k1 + 0xBB67AE85u);
    const uint32_t m3 = (uint32_t)q0;
    const uint64_t r1 = (uint64_t)0xCD9E8D57u * (uint64_t)m2;
    uint32_t c0 = (uint32_t)(r1 >> 32) ^ f.m1 ^ (f.k0 + 2u * 0x9E3779B9u);
    uint32_t cc1 = (uint32_t)r1;
    uint32_t c2 = f.hp0 ^ m3 ^ (f.k1 + 2u * 0xBB67AE85u);
    uint32_t c3 = f.o3;
    uint32_t k0 = f.k0 + 3u * 0x9E3779B9u, k1 = f.k1 + 3u * 0xBB67AE85u;
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t a0 = (uint32_t)(p1 >> 32) ^ cc1 ^ k0;
        const uint32_t a2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        cc1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = a0;
        c2 = a2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, cc1, c2, c3);
}

// Full Philox4x32-10 with the round keys read from arrays.
__device__ __forceinline__ uint4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           const uint32_t *rk0, const uint32_t *rk1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

// The same with the ten round keys of each key word read from arrays (kernel parameters:
// constant-bank operands of the XORs, nothing recomputed per call).
__device__ __forceinline__ PhiloxPrefix philox_prefix_rk(uint32_t c0, uint32_t c2, uint32_t c3,
                                                         const uint32_t *rk0, const uint32_t *rk1) {
    PhiloxPrefix f;
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    f.x0 = (uint32_t)(p1 >> 32) ^ rk0[0];
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[0];
    f.n3 = (uint32_t)p0;
    const uint64_t q1 = (uint64_t)0xCD9E8D57u * (uint64_t)n2;
    f.m0 = (uint32_t)(q1 >> 32) ^ n1 ^ rk0[1];
    f.m1 = (uint32_t)q1;
    const uint64_t r0 = (uint64_t)0xD2511F53u * (uint64_t)f.m0;
    f.hp0 = (uint32_t)(r0 >> 32);
    f.o3 = (uint32_t)r0;
    f.k0 = rk0[0];
    f.k1 = rk1[0];
    return f;
}

__device__ __forceinline__ uint4 philox_from_prefix_rk(const PhiloxPrefix &f, uint32_t c1,
                                                       const uint32_t *rk0, const uint32_t *rk1) {
    const uint32_t n0 = f.x0 ^ c1;
    const uint64_t q0 = (uint64_t)0xD2511F53u * (uint64_t)n0;
    const uint32_t m2 = (uint32_t)(q0 >> 32) ^ f.n3 ^ rk1[1];
    const uint32_t m3 = (uint32_t)q0;
    const uint64_t r1 = (uint64_t)0xCD9E8D57u * (uint64_t)m2;
    uint32_t c0 = (uint32_t)(r1 >> 32) ^ f.m1 ^ rk0[2];
    uint32_t cc1 = (uint32_t)r1;
    uint32_t c2 = f.hp0 ^ m3 ^ rk1[2];
    uint32_t c3 = f.o3;
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t a0 = (uint32_t)(p1 >> 32) ^ cc1 ^ rk0[r];
        const uint32_t a2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
        cc1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = a0;
        c2 = a2;
    }
    return make_uint4(c0, cc1, c2, c3);
}

__device__ __forceinline__ uint32_t rng_tag(uint32_t kind, uint32_t half, uint32_t sub) {
    return (kind << 28) | (half << 27) | sub;
}

// u(w) = ((w >> 8) | 1) * 2^-24: exact in FP32, in (0, 1).
__device__ __forceinline__ float uniform_of(uint32_t w) {
    return __fmul_rn(__uint2float_rn((w >> 8) | 1u), 5.9604644775390625e-08f);
}

__device__ __forceinline__ uint32_t word_of(const uint4 &w, uint32_t k) {
    return k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
}

// Draw-word parts of inversion point i: the coarse byte is byte i & 3 of word (i & 15) >> 2 of
// the HI call of group i >> 4; the low 24 bits are the top 24 bits of word i & 3 of the LO call
// of quad i >> 2.  x = byte << 24 | low24.
__device__ __forceinline__ uint32_t hi_byte(const uint4 &w, uint32_t j) {
    return (word_of(w, j >> 2) >> (8u * (j & 3u))) & 0xFFu;
}

// ---------------------------------------------------------------------------------------
// FP32 natural log from IEEE basic operations (every operation round-to-nearest, never
// contracted): exponent split, mantissa in [sqrt(1/2), sqrt(2)], and the atanh series
// ln m = 2 (s + s^3/3 + ... + s^11/11), s = (m - 1) / (m + 1) (Abramowitz & Stegun 4.1.27).
// Finite normal x > 0 only.  Used wherever a logarithm decides a star count.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float ln_series(float x) {
    const float kLn2Hi = 0.693145751953125f;  // 45426 / 2^16: e * kLn2Hi is exact
    const float kLn2Lo = (float)(0.69314718055994530942 - 0.693145751953125);
    const float k3 = (float)(1.0 / 3.0), k5 = (float)(1.0 / 5.0), k7 = (float)(1.0 / 7.0);
    const float k9 = (float)(1.0 / 9.0), k11 = (float)(1.0 / 11.0);
    const uint32_t u = __float_as_uint(x);
    int e = (int)(u >> 23) - 127;
    float m = __uint_as_float((u & 0x007FFFFFu) | 0x3F800000u);
    if (m > __uint_as_float(0x3FB504F3u)) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float z = __fmul_rn(s, s);
    float p = k11;
    p = __fadd_rn(__fmul_rn(p, z), k9);
    p = __fadd_rn(__fmul_rn(p, z), k7);
    p = __fadd_rn(__fmul_rn(p, z), k5);
    p = __fadd_rn(__fmul_rn(p, z), k3);
    const float t = __fmul_rn(__fmul_rn(s, z), p);
    float lnm = __fadd_rn(s, t);
    lnm = __fadd_rn(lnm, lnm);
    const float ef = __int2float_rn(e);
    return __fadd_rn(__fadd_rn(lnm, __fmul_rn(ef, kLn2Lo)), __fmul_rn(ef, kLn2Hi));
}

// phi(x) = (1+x) ln(1+x) - x: alternating series sum_{n=2}^{13} (-1)^n x^n / (n(n-1)) for
// |x| < 1/4 (Horner from the x^13 coefficient), else the closed form with ln_series.
__device__ __forceinline__ float phi_dev(float x) {
    if (fabsf(x) < 0.25f) {
        float p = (float)(-1.0 / (13.0 * 12.0));
        p = __fadd_rn(__fmul_rn(p, x), (float)(1.0 / (12.0 * 11.0)));
        p = __fadd_rn(__fmul_rn(p, x), (float)(-1.0 / (11.0 * 10.0)));
        p = __fadd_rn(__fmul_rn(p, x), (float)(1.0 / (10.0 * 9.0)));
        p = __fadd_rn(__fmul_rn(p, x), (float)(-1.0 / (9.0 * 8.0)));
        p = __fadd_rn(__fmul_rn(p, x), (float)(1.0 / (8.0 * 7.0)));
        p = __fadd_rn(__fmul_rn(p, x), (float)(-1.0 / (7.0 * 6.0)));
        p = __fadd_rn(__fmul_rn(p, x), (float)(1.0 / (6.0 * 5.0)));
        p = __fadd_rn(__fmul_rn(p, x), (float)(-1.0 / (5.0 * 4.0)));
        p = __fadd_rn(__fmul_rn(p, x), (float)(1.0 / (4.0 * 3.0)));
        p = __fadd_rn(__fmul_rn(p, x), (float)(-1.0 / (3.0 * 2.0)));
        p = __fadd_rn(__fmul_rn(p, x), (float)(1.0 / (2.0 * 1.0)));
        return __fmul_rn(__fmul_rn(p, x), x);
    }
    const float y = __fadd_rn(1.0f, x);
    return __fsub_rn(__fmul_rn(y, ln_series(y)), x);
}

// ---------------------------------------------------------------------------------------
// Bulk-copy staging (cp.async.bulk + mbarrier) with waits bounded in wall time.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_arrive_local(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity; gives up after ~2 s, latching kErrTimeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t *err) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > 2000000000ull) {
            atomicOr(err, kErrTimeout);
            return false;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Pixel stage: sky + photon noise, magnitudes, colour and the FP32 Hess bin rule.
// ---------------------------------------------------------------------------------------
struct PixelOut {
    float mag, col;
    int bin;        // -1 = outside the grid
    bool valid;
};

// FP32 Hess bin rule: ix = floor((colour - c_lo) * inv_w), iy = floor((mag - m_lo) * inv_w);
// bin = iy * nx + ix inside the grid, -1 outside.
__device__ __forceinline__ int hess_bin(float mag, float col, const PixelConsts &pc) {
    const float fx = floorf(__fmul_rn(__fsub_rn(col, pc.c_lo), pc.inv_w));
    const float fy = floorf(__fmul_rn(__fsub_rn(mag, pc.m_lo), pc.inv_w));
    if (fx >= 0.0f && fx < (float)pc.nx && fy >= 0.0f && fy < (float)pc.ny)
        return (int)fy * pc.nx + (int)fx;
    return -1;
}

template <int B>
__device__ __forceinline__ PixelOut pixel_stage(float (&F)[B], uint32_t pix, uint32_t set,
                                                const PixelConsts &pc) {
    if (pc.noise) {
        const uint32_t k0 = (uint32_t)pc.seed, k1 = (uint32_t)(pc.seed >> 32);
#pragma unroll
        for (int q = 0; q < (B + 1) / 2; ++q) {
            const uint4 w = philox(pix, (uint32_t)q, set, rng_tag(kKindNoise, 0, 0), k0, k1);
            const float u1 = uniform_of(w.x), u2 = uniform_of(w.y);
            const float r = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
            const float z[2] = {r * cs, r * sn};
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int b = 2 * q + t;
                if (b < B) F[b] = F[b] + sqrtf(fmaxf(F[b] + pc.sky[b], 0.0f)) * z[t];
            }
        }
    }
    PixelOut o;
    o.valid = F[0] > 0.0f && F[1] > 0.0f;
    o.bin = -1;
    o.mag = 0.0f;
    o.col = 0.0f;
    if (o.valid) {
        // m_b = ZP_b - 2.5 log10(F_b / t_b); ZP split in hi + lo parts to keep FP32 accuracy
        const float l0 = log10f(__fdiv_rn(F[0], pc.t[0]));
        const float l1 = log10f(__fdiv_rn(F[1], pc.t[1]));
        const float m0 = __fadd_rn(pc.zp[0], fmaf(-2.5f, l0, pc.zp_lo[0]));
        const float m1 = __fadd_rn(pc.zp[1], fmaf(-2.5f, l1, pc.zp_lo[1]));
        o.mag = m0;
        o.col = __fsub_rn(m1, m0);
        o.bin = hess_bin(o.mag, o.col, pc);
    }
    return o;
}

// Warp-aggregated shared-memory histogram increment: lanes hitting the same bin elect one
// leader that adds the group's population.  Records a bin in `touched` on its first hit.
__device__ __forceinline__ void hist_add_warp(uint32_t *hist, uint32_t *touched,
                                              uint32_t *n_touched, int bin, uint32_t cap) {
    const uint32_t active = __activemask();
    const uint32_t peers = __match_any_sync(active, bin);
    const int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader && bin >= 0) {
        const uint32_t old = atomicAdd(&hist[bin], (uint32_t)__popc(peers));
        if (old == 0u && touched != nullptr) {
            const uint32_t slot = atomicAdd(n_touched, 1u);
            if (slot < cap) touched[slot] = (uint32_t)bin;
        }
    }
}

}  // namespace pcmd
