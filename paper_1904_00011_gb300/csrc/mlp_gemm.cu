// BF16 GEMM on the fifth-generation tensor cores: C = epilogue(A[M,K] . B[N,K]^T), FP32
// accumulation in tensor memory.
//
// Persistent kernel, one CTA (18 warps) per SM, 128 x 256 output tiles taken in a fixed
// stride over the tile list.  Warp 0 (one lane) streams 128x64 / 256x64 K-major tiles of A and
// B into a 4-stage shared-memory ring with TMA (128-byte swizzle); warp 1 owns the tensor
// memory (two 256-column FP32 accumulators) and one of its lanes issues tcgen05.mma (M=128,
// N=256, K=16 per instruction), committing each stage back to the producer and each finished
// tile to the epilogue; warps 2-17 (four per TMEM lane quarter, one per 64-column block) read
// their accumulator rows with tcgen05.ld, apply the epilogue, stage 32 x 32 blocks in swizzled
// shared memory and write them with TMA stores (whole rows per transaction, edges clipped by
// the tensor map), then hand the accumulator back.  With two accumulators the epilogue of one
// tile overlaps the main loop of the next.  Every mbarrier
// wait is bounded in wall time; a wait that runs out latches an error, the roles drain what
// they have in flight (TMA copies, MMAs) and the CTA frees its tensor memory before it exits.
#include <cuda.h>
#include <cstring>
#include <cuda_bf16.h>

#include "common.cuh"
#include "mlp_internal.h"

namespace pcmd {

constexpr int kGemmBM = 128;
constexpr int kGemmBN = kGemmTileN;
constexpr int kGemmBK = 64;          // 64 BF16 = 128 bytes: one swizzle row
constexpr int kGemmStages = 4;
constexpr int kGemmEpiWarps = 4 * kGemmLlBlocks;           // four per TMEM lane quarter
constexpr int kGemmEpiCols = kGemmBN / kGemmLlBlocks;      // columns of one epilogue warp
constexpr int kGemmThreads = 64 + 32 * kGemmEpiWarps;
constexpr uint32_t kGemmStageOut = 2048;   // per epilogue warp: one 32-row x 64-byte output block

// ---- tcgen05 / TMA primitives (inline PTX) -------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 128 bytes,
// 8-row swizzle atoms 1024 bytes apart (stride byte offset), start address >> 4.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;                       // leading byte offset (unused for this layout)
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;  // stride byte offset
    d |= (uint64_t)1u << 46;                       // descriptor version
    d |= (uint64_t)2u << 61;                       // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, with erfc(x) = P(t) exp(-x^2), t = 1 / (1 + p x)
// for x >= 0 (Abramowitz & Stegun 7.1.26, |error of erf| <= 1.5e-7): z >= 0 gives
// z - z erfc / 2, z < 0 gives z erfc(|z| / sqrt 2) / 2 with no cancellation.  The output is
// rounded to BF16, whose spacing is far above this error.
__device__ __forceinline__ float gelu_f(float z) {
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    float p = 1.061405429f;
    p = fmaf(p, t, -1.453152027f);
    p = fmaf(p, t, 1.421413741f);
    p = fmaf(p, t, -0.284496736f);
    p = fmaf(p, t, 0.254829592f);
    const float erfc_x = p * t * __expf(-x * x);
    const float h = 0.5f * z * erfc_x;
    return z >= 0.0f ? z - h : h;
}

struct GemmLayout {
    static constexpr uint32_t a_bytes = kGemmBM * kGemmBK * 2;
    static constexpr uint32_t b_bytes = kGemmBN * kGemmBK * 2;
    static constexpr uint32_t stage_bytes = a_bytes + b_bytes;
    static constexpr uint32_t out_off = kGemmStages * stage_bytes;            // 1024-aligned
    static constexpr uint32_t bar_off = out_off + kGemmEpiWarps * kGemmStageOut;
    static constexpr size_t smem = 1024 + (size_t)bar_off + 256;
};

// Epilogue of 16 consecutive columns [col0, col0 + 16) of one row.
template <int EPI>
__device__ __forceinline__ void epilogue16(const GemmArgs &g, int row, int col0, float (&v)[16], bool vec) {
    if (row >= g.m || col0 >= g.n) return;
    const bool full16 = col0 + 16 <= g.n;
    if (EPI != kEpiF32) {
        if (full16 && vec) {
            const float4 *b4 = reinterpret_cast<const float4 *>(g.bias + col0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 b = __ldg(b4 + j);
                v[4 * j] += b.x;
                v[4 * j + 1] += b.y;
                v[4 * j + 2] += b.z;
                v[4 * j + 3] += b.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (col0 + j < g.n) v[j] += __ldg(g.bias + col0 + j);
        }
    }
    if (EPI == kEpiF32 || EPI == kEpiBiasF32) {
        float *out = reinterpret_cast<float *>(g.c) + (size_t)row * g.ldc + col0;
        if (full16 && vec) {
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4 *>(out + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (col0 + j < g.n) out[j] = v[j];
        }
        return;
    }
    __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(g.c) + (size_t)row * g.ldc + col0;
    __nv_bfloat16 *aux = EPI == kEpiBiasGeluBf16 && g.aux
                             ? reinterpret_cast<__nv_bfloat16 *>(g.aux) + (size_t)row * g.ldc + col0
                             : nullptr;
    if (full16 && vec) {
        uint32_t po[8], pa[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float z0 = v[2 * j], z1 = v[2 * j + 1];
            __nv_bfloat162 zb = __floats2bfloat162_rn(z0, z1);
            pa[j] = *reinterpret_cast<uint32_t *>(&zb);
            if (EPI == kEpiBiasGeluBf16) {
                __nv_bfloat162 gb = __floats2bfloat162_rn(gelu_f(z0), gelu_f(z1));
                po[j] = *reinterpret_cast<uint32_t *>(&gb);
            } else {
                po[j] = pa[j];
            }
        }
        uint4 *o4 = reinterpret_cast<uint4 *>(out);
        o4[0] = make_uint4(po[0], po[1], po[2], po[3]);
        o4[1] = make_uint4(po[4], po[5], po[6], po[7]);
        if (EPI == kEpiBiasGeluBf16 && aux) {
            uint4 *a4 = reinterpret_cast<uint4 *>(aux);
            a4[0] = make_uint4(pa[0], pa[1], pa[2], pa[3]);
            a4[1] = make_uint4(pa[4], pa[5], pa[6], pa[7]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (col0 + j >= g.n) continue;
            if (EPI == kEpiBiasGeluBf16) {
                if (aux) aux[j] = __float2bfloat16_rn(v[j]);
                out[j] = __float2bfloat16_rn(gelu_f(v[j]));
            } else {
                out[j] = __float2bfloat16_rn(v[j]);
            }
        }
    }
}

template <int EPI>
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_bf16_kernel(const __grid_constant__ CUtensorMap tm_a,
                                                                    const __grid_constant__ CUtensorMap tm_b,
                                                                    const __grid_constant__ CUtensorMap tm_c,
                                                                    const __grid_constant__ CUtensorMap tm_aux,
                                                                    const GemmArgs g) {
    using L = GemmLayout;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    uint8_t *tiles = base;
    uint8_t *out_stage = base + L::out_off;
    uint64_t *full = reinterpret_cast<uint64_t *>(base + L::bar_off);
    uint64_t *empty = full + kGemmStages;
    uint64_t *tfull = empty + kGemmStages;     // [2] accumulator ready for the epilogue
    uint64_t *tempty = tfull + 2;              // [2] accumulator drained by the epilogue
    uint64_t *done = tempty + 2;               // all MMAs of this CTA complete
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile uint32_t *abort_flag = tmem_slot + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kGemmStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 32 * kGemmEpiWarps);
        }
        mbar_init(done, 1);
        *abort_flag = 0u;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, 2 * kGemmBN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tmem_slot;

    const int n_m = (g.m + kGemmBM - 1) / kGemmBM;
    const int n_n = (g.n + kGemmBN - 1) / kGemmBN;
    const int n_tiles = n_m * n_n;
    const int nk = (g.k + kGemmBK - 1) / kGemmBK;
    constexpr uint32_t idesc = idesc_bf16(kGemmBM, kGemmBN);

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            uint32_t kc = 0;   // k blocks issued by this CTA
            for (int t = blockIdx.x; t < n_tiles && !*abort_flag; t += gridDim.x) {
                const int m0 = (t % n_m) * kGemmBM, n0 = (t / n_m) * kGemmBN;
                for (int kb = 0; kb < nk; ++kb, ++kc) {
                    const uint32_t s = kc % kGemmStages, use = kc / kGemmStages;
                    if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1u, g.err)) {
                        *abort_flag = 1u;
                        break;
                    }
                    uint8_t *sa = tiles + s * L::stage_bytes;
                    mbar_expect_tx(&full[s], L::stage_bytes);
                    tma_load_2d(sa, &tm_a, kb * kGemmBK, m0, &full[s]);
                    tma_load_2d(sa + L::a_bytes, &tm_b, kb * kGemmBK, n0, &full[s]);
                }
            }
            // drain: the copies of the last issued stages have landed before the CTA exits
            const uint32_t first = kc > (uint32_t)kGemmStages ? kc - kGemmStages : 0u;
            for (uint32_t c = first; c < kc; ++c)
                mbar_wait(&full[c % kGemmStages], (c / kGemmStages) & 1u, g.err);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            uint32_t kc = 0, it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++it) {
                const uint32_t buf = it & 1u, use = it >> 1;
                if (use > 0 && !mbar_wait(&tempty[buf], (use - 1) & 1u, g.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = taddr + buf * kGemmBN;
                for (int kb = 0; kb < nk; ++kb, ++kc) {
                    const uint32_t s = kc % kGemmStages;
                    if (*abort_flag || !mbar_wait(&full[s], (kc / kGemmStages) & 1u, g.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(tiles + s * L::stage_bytes);
                    const uint32_t sb = sa + L::a_bytes;
#pragma unroll
                    for (int kk = 0; kk < kGemmBK / 16; ++kk)
                        umma_bf16(d, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), idesc,
                                  (kb | kk) != 0 ? 1u : 0u);
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&tfull[buf]);
            }
            if (!ok) *abort_flag = 1u;
            umma_commit(done);
            mbar_wait(done, 0u, g.err);
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns 128 h .. + 127 ----
        const uint32_t q = (uint32_t)(warp & 3);
        const int h = (warp - 2) >> 2;      // column block of this warp
        uint8_t *stage = out_stage + (warp - 2) * kGemmStageOut;
        const bool vec = ((g.ldc & 7) == 0) && ((reinterpret_cast<uintptr_t>(g.c) & 15) == 0) &&
                         (EPI != kEpiBiasGeluBf16 || (reinterpret_cast<uintptr_t>(g.aux) & 15) == 0) &&
                         (EPI == kEpiF32 || (reinterpret_cast<uintptr_t>(g.bias) & 15) == 0);
        const bool aux_on = EPI == kEpiBiasGeluBf16 && g.aux != nullptr;
        uint32_t it = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
            const uint32_t buf = it & 1u, use = it >> 1;
            int ready = 0;
            if (lane == 0) ready = !*abort_flag && mbar_wait(&tfull[buf], use & 1u, g.err);
            ready = __shfl_sync(0xffffffffu, ready, 0);
            if (!ready) {
                *abort_flag = 1u;
                break;
            }
            tc_fence_after();
            const int m0 = (t % n_m) * kGemmBM, n0 = (t / n_m) * kGemmBN;
            const int rbase = m0 + (int)(q * 32);
            const uint32_t tbase = taddr + ((q * 32u) << 16) + buf * kGemmBN + (uint32_t)(h * kGemmEpiCols);
            double ll_acc = 0.0;
#pragma unroll 1
            for (int c = 0; c < kGemmEpiCols; c += 32) {
                uint32_t r0[16], r1[16];
                tmem_ld16_nowait(tbase + (uint32_t)c, r0);
                tmem_ld16_nowait(tbase + (uint32_t)c + 16u, r1);
                tmem_ld_wait();
                if (c == kGemmEpiCols - 32) {   // the accumulator is no longer read: hand it back
                    tc_fence_before();
                    mbar_arrive_local(&tempty[buf]);
                }
                float v[32];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = __uint_as_float(r0[j]);
                    v[16 + j] = __uint_as_float(r1[j]);
                }
                const int col0 = n0 + h * kGemmEpiCols + c;
                if (EPI == kEpiPoissonLL) {
                    float sum = 0.0f;
                    if (col0 + 32 <= g.n) {
                        const float4 *b4 = reinterpret_cast<const float4 *>(g.bias + col0);
                        const uint4 *d4 = reinterpret_cast<const uint4 *>(g.ll_data + col0);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float4 bb = __ldg(b4 + j);
                            const uint4 dd = __ldg(d4 + j);
                            sum += surrogate_ll_term(v[4 * j] + bb.x, dd.x, g.llk, g.ll_poisson);
                            sum += surrogate_ll_term(v[4 * j + 1] + bb.y, dd.y, g.llk, g.ll_poisson);
                            sum += surrogate_ll_term(v[4 * j + 2] + bb.z, dd.z, g.llk, g.ll_poisson);
                            sum += surrogate_ll_term(v[4 * j + 3] + bb.w, dd.w, g.llk, g.ll_poisson);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (col0 + j < g.n)
                                sum += surrogate_ll_term(v[j] + __ldg(g.bias + col0 + j), __ldg(g.ll_data + col0 + j),
                                                         g.llk, g.ll_poisson);
                    }
                    ll_acc += (double)sum;
                    continue;
                }
                if (!g.tma_store) {
                    float va[16], vb[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        va[j] = v[j];
                        vb[j] = v[16 + j];
                    }
                    epilogue16<EPI>(g, rbase + lane, col0, va, vec);
                    epilogue16<EPI>(g, rbase + lane, col0 + 16, vb, vec);
                    continue;
                }
                if (col0 >= g.n) continue;    // warp-uniform: nothing of this block is inside
                if (EPI != kEpiF32) {
                    if (col0 + 32 <= g.n) {
                        const float4 *b4 = reinterpret_cast<const float4 *>(g.bias + col0);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float4 bb = __ldg(b4 + j);
                            v[4 * j] += bb.x;
                            v[4 * j + 1] += bb.y;
                            v[4 * j + 2] += bb.z;
                            v[4 * j + 3] += bb.w;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (col0 + j < g.n) v[j] += __ldg(g.bias + col0 + j);
                    }
                }
                // Staging: 32 rows x 64 bytes with 64-byte swizzle (16-byte unit u of row r at
                // u ^ ((r >> 1) & 3)); FP32 goes out as two 16-column blocks, BF16 as one
                // 32-column block (then the pre-activations through the same buffer).
                uint8_t *row = stage + lane * 64;
                const int sw = (lane >> 1) & 3;
                if (EPI == kEpiF32 || EPI == kEpiBiasF32) {
#pragma unroll
                    for (int sb = 0; sb < 2; ++sb) {
                        if (lane == 0) bulk_wait_read0();   // the previous block left the buffer
                        __syncwarp();
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            *reinterpret_cast<float4 *>(row + ((u ^ sw) << 4)) =
                                make_float4(v[16 * sb + 4 * u], v[16 * sb + 4 * u + 1], v[16 * sb + 4 * u + 2],
                                            v[16 * sb + 4 * u + 3]);
                        fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0 && col0 + 16 * sb < g.n) {
                            tma_store_2d(&tm_c, stage, col0 + 16 * sb, rbase);
                            bulk_commit();
                        }
                    }
                } else {
                    uint32_t po[16], pa[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float z0 = v[2 * j], z1 = v[2 * j + 1];
                        __nv_bfloat162 zb = __floats2bfloat162_rn(z0, z1);
                        pa[j] = *reinterpret_cast<uint32_t *>(&zb);
                        if (EPI == kEpiBiasGeluBf16) {
                            __nv_bfloat162 gb = __floats2bfloat162_rn(gelu_f(z0), gelu_f(z1));
                            po[j] = *reinterpret_cast<uint32_t *>(&gb);
                        } else {
                            po[j] = pa[j];
                        }
                    }
                    if (lane == 0) bulk_wait_read0();
                    __syncwarp();
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        *reinterpret_cast<uint4 *>(row + ((u ^ sw) << 4)) =
                            make_uint4(po[4 * u], po[4 * u + 1], po[4 * u + 2], po[4 * u + 3]);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&tm_c, stage, col0, rbase);
                        bulk_commit();
                    }
                    if (aux_on) {
                        if (lane == 0) bulk_wait_read0();
                        __syncwarp();
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            *reinterpret_cast<uint4 *>(row + ((u ^ sw) << 4)) =
                                make_uint4(pa[4 * u], pa[4 * u + 1], pa[4 * u + 2], pa[4 * u + 3]);
                        fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            tma_store_2d(&tm_aux, stage, col0, rbase);
                            bulk_commit();
                        }
                    }
                }
            }
            if (EPI == kEpiPoissonLL && rbase + lane < g.m)
                g.ll_part[(size_t)(rbase + lane) * g.ll_ld + (t / n_m) * kGemmLlBlocks + h] = ll_acc;
        }
        if (lane == 0) bulk_wait0();
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(taddr, 2 * kGemmBN);
}

// ---- host side --------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D BF16 tensor map of a row-major [rows][ld] matrix with `cols` valid columns, box 64 x box_rows.
static bool make_map(CUtensorMap *map, const void *ptr, int rows, int cols, int ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kGemmBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D tensor map of an output [rows][ld] (FP32 or BF16) written in blocks of 32 rows x 64
// bytes (16 FP32 or 32 BF16 columns) with 64-byte swizzle.
static bool make_store_map(CUtensorMap *map, void *ptr, int rows, int cols, int ld, bool bf16) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const size_t es = bf16 ? 2 : 4;
    if (((uintptr_t)ptr & 15) || ((size_t)ld * es) % 16) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * es};
    cuuint32_t box[2] = {(cuuint32_t)(64 / es), 32};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims,
              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int EPI>
static cudaError_t launch_t(const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap &tc,
                            const CUtensorMap &taux, const GemmArgs &g, cudaStream_t st) {
    using L = GemmLayout;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel<EPI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm <= 0)
            n_sm = 1;
    }
    const int tiles = ((g.m + kGemmBM - 1) / kGemmBM) * ((g.n + kGemmBN - 1) / kGemmBN);
    gemm_bf16_kernel<EPI><<<tiles < n_sm ? tiles : n_sm, kGemmThreads, L::smem, st>>>(ta, tb, tc, taux, g);
    return cudaGetLastError();
}

cudaError_t launch_gemm_bf16(const void *a, int lda, const void *b, int ldb, const GemmArgs &g,
                             int epilogue, cudaStream_t st) {
    if (g.m <= 0 || g.n <= 0 || g.k <= 0 || (lda & 7) || (ldb & 7) || lda < g.k || ldb < g.k ||
        ((uintptr_t)a & 15) || ((uintptr_t)b & 15) || !g.err)
        return cudaErrorInvalidValue;
    if (epilogue < kEpiF32 || epilogue > kEpiPoissonLL) return cudaErrorInvalidValue;
    if (epilogue != kEpiF32 && !g.bias) return cudaErrorInvalidValue;
    CUtensorMap ta, tb, tc, taux;
    if (!make_map(&ta, a, g.m, g.k, lda, kGemmBM) || !make_map(&tb, b, g.n, g.k, ldb, kGemmBN))
        return cudaErrorInvalidValue;
    GemmArgs gg = g;
    std::memset(&tc, 0, sizeof tc);
    std::memset(&taux, 0, sizeof taux);
    if (epilogue == kEpiPoissonLL) {
        const int n_n = (g.n + kGemmBN - 1) / kGemmBN;
        if (!g.ll_data || !g.ll_part || g.ll_ld < kGemmLlBlocks * n_n || ((uintptr_t)g.ll_data & 15) ||
            ((uintptr_t)g.bias & 15))
            return cudaErrorInvalidValue;
        gg.tma_store = 0;
        return launch_t<kEpiPoissonLL>(ta, tb, tc, taux, gg, st);
    }
    if (g.ldc < g.n || !g.c) return cudaErrorInvalidValue;
    const bool bf16 = epilogue == kEpiBiasGeluBf16 || epilogue == kEpiBiasBf16;
    gg.tma_store = make_store_map(&tc, g.c, g.m, g.n, g.ldc, bf16) &&
                   (epilogue != kEpiBiasGeluBf16 || !g.aux || make_store_map(&taux, g.aux, g.m, g.n, g.ldc, true));
    switch (epilogue) {
        case kEpiF32: return launch_t<kEpiF32>(ta, tb, tc, taux, gg, st);
        case kEpiBiasF32: return launch_t<kEpiBiasF32>(ta, tb, tc, taux, gg, st);
        case kEpiBiasGeluBf16: return launch_t<kEpiBiasGeluBf16>(ta, tb, tc, taux, gg, st);
        default: return launch_t<kEpiBiasBf16>(ta, tb, tc, taux, gg, st);
    }
}

}  // namespace pcmd
