// Shared-memory layout, warp roles and barrier helpers of the tcgen05 update kernels (the
// per-launch update kernel in k_tc.cu and the persistent stage kernel in k_stage.cu).
#pragma once

#include "common.cuh"
#include "internal.h"

namespace ica {

// Samples per chunk and number of Z / P buffers: with NB buffers the first product runs up to
// NB chunks ahead of the epilogue, so the cube conversion of one chunk overlaps the products of
// the next ones. TMEM holds D2 (n_pad columns) plus NB Z buffers of TC columns;
// shared memory must keep at least NB + 1 X~ stages in flight (NB stages are pinned by chunks
// waiting for their second product).
// Chunks are as wide as TMEM and shared memory allow (fixed costs per chunk - barrier round
// trips and commits - dominate at small n): n_pad <= 64 uses 192 samples (accumulator 64
// columns + 2 x 192), n_pad <= 128 uses 128 (128 + 2 x 128 columns; three 32 KB X~ stages),
// larger n_pad 64.
#ifndef ICA_TC_SMALL_CHUNK
#define ICA_TC_SMALL_CHUNK 192
#endif
#ifndef ICA_TC_SMALL_NB
#define ICA_TC_SMALL_NB 2
#endif
// Restart rows as two BF16 terms (hi = bf16(b), lo = bf16(b - hi)) in the first product: Z =
// B_hi X~ + B_lo X~ carries b to about 16 bits instead of 8, so that the BF16 stage's step
// distance can fall below its tolerance instead of stalling at the rounding noise of b (without
// it, at n_pad > 64 no restart of the EEG-like N = 128 and N = 256 workloads converged: every one
// ran all iterations). Costs one more MMA per K step of the first product. Where the two tiles
// fit shared memory (192-sample chunks, n_pad <= 64) lo sits beside hi there; for 128- and
// 64-sample chunks lo goes to tensor memory (n_pad / 2 columns after the Z buffers) and the
// first product reads it as a TMEM A operand.
#ifndef ICA_TC_SPLIT_B
#define ICA_TC_SPLIT_B 1
#endif
__host__ __device__ constexpr bool tc_split_b(int TC) { return ICA_TC_SPLIT_B != 0; }
__host__ __device__ constexpr bool tc_lo_in_tmem(int TC) { return ICA_TC_SPLIT_B != 0 && TC != 192; }
// Second products issued by two threads (on different schedulers) into two accumulators, summed
// when read out: measured on GB300, one thread sustained one M128 K16 MMA per 67 cycles at
// N <= 64 and two threads one per 50 (N = 64) or 41 (N = 16) cycles. Both accumulators fit TMEM
// next to the Z buffers for TC = 192 (n_pad <= 64); for TC = 128 only while B's low term does not
// occupy TMEM (at N = 128 one issuing thread is close to the execution rate of the MMA).
__host__ __device__ constexpr int tc_g2_issuers(int TC) {
    return TC == 192 ? 2 : (TC == 128 && !tc_lo_in_tmem(128) ? 2 : 1);
}
__host__ __device__ constexpr uint32_t tc_d2_cols(int TC) { return TC == 192 ? 64u : (TC == 128 ? 128u : 256u); }
// First TMEM column of B's low term (after the G2S accumulators and the NB Z buffers).
__host__ __device__ constexpr uint32_t tc_alo_col(int TC, int NB) {
    return static_cast<uint32_t>(tc_g2_issuers(TC)) * tc_d2_cols(TC) + static_cast<uint32_t>(NB * TC);
}

namespace {
constexpr int kBars = 40;
#ifndef ICA_TC_EPI_WARPS
#define ICA_TC_EPI_WARPS 16
#endif
constexpr int kEpiWarps = ICA_TC_EPI_WARPS;  // 4 lane quarters x kEpiWarps / 4 column groups
constexpr int kGroups = kEpiWarps / 4;
static_assert(kEpiWarps == 8 || kEpiWarps == 16, "two or four column groups");
constexpr int kG2Warp = 2 + kEpiWarps;   // issues the second products (even K steps)
constexpr int kG2bWarp = 3 + kEpiWarps;  // issues their odd K steps when the issue is split
constexpr int kThreads = 32 * (4 + kEpiWarps);
constexpr uint32_t kScratchBytes = 8192u;  // barriers, TMEM slot, moment exchange
struct TcLayout {
    uint32_t a_bytes, xsub_bytes, xstage_bytes, p_bytes, stages, off_x, off_p, off_bar, total;
};
// reserve: bytes of the 227 KB per-CTA shared memory left for the kernel's static shared memory
TcLayout tc_layout(int n_pad, bool moments_only, int TC, int NB, uint32_t reserve = 0) {
    TcLayout L{};
    L.a_bytes = static_cast<uint32_t>((n_pad + 63) / 64) * 16384u * (tc_split_b(TC) && !tc_lo_in_tmem(TC) ? 2u : 1u);
    L.xsub_bytes = static_cast<uint32_t>(n_pad) * 128u;
    L.xstage_bytes = static_cast<uint32_t>(TC / 64) * L.xsub_bytes;  // X~ tile: n_pad rows x TC samples
    L.p_bytes = moments_only ? 0u : static_cast<uint32_t>(TC / 64) * 16384u;
    const uint32_t fixed = L.a_bytes + NB * L.p_bytes + kScratchBytes + 1024u;  // + scratch + alignment
    const uint32_t budget = 227u * 1024u - reserve;
    uint32_t st = (budget - fixed) / L.xstage_bytes;
    if (st > 8) st = 8;
    L.stages = st;
    L.off_x = L.a_bytes;
    L.off_p = L.off_x + st * L.xstage_bytes;
    L.off_bar = L.off_p + NB * L.p_bytes;
    L.total = L.off_bar + kScratchBytes + 1024u;
    // one CTA per SM: the kernel allocates all 512 TMEM columns
    if (L.total < 120u * 1024u) L.total = 120u * 1024u;
    return L;
}
// Layout of the FP8 stage (E4M3 operands, 128-sample chunks): the restart tile as two E4M3 terms
// (hi, then lo in the second half of the region; each K-major, 128-byte swizzle, K blocks of 128
// entries at 16 KB), X~ stages of n8 rows x 128
// samples (one byte each: the TMA box {128, n8}), two P tiles of 128 x 128 bytes. n8 = the reduced
// dimension rounded up to 32 (the K of one E4M3 MMA). The restart-tile region doubles as the row
// completion's scratch, so it is at least 16 warps x (2 n_pad + 4) floats.
TcLayout tc_layout_e4m3(int n8, int n_pad, uint32_t reserve = 0) {
    TcLayout L{};
    uint32_t a = 2u * static_cast<uint32_t>((n8 + 127) / 128) * 16384u;
    const uint32_t fin = (16u * static_cast<uint32_t>(2 * n_pad + 4) * 4u + 2047u) & ~2047u;  // halves 1 KB aligned
    L.a_bytes = a > fin ? a : fin;
    L.xsub_bytes = static_cast<uint32_t>(n8) * 128u;
    L.xstage_bytes = L.xsub_bytes;
    L.p_bytes = 16384u;
    const uint32_t fixed = L.a_bytes + 2u * L.p_bytes + kScratchBytes + 1024u;
    const uint32_t budget = 227u * 1024u - reserve;
    uint32_t st = (budget - fixed) / L.xstage_bytes;
    if (st > 8) st = 8;
    L.stages = st;
    L.off_x = L.a_bytes;
    L.off_p = L.off_x + st * L.xstage_bytes;
    L.off_bar = L.off_p + 2u * L.p_bytes;
    L.total = L.off_bar + kScratchBytes + 1024u;
    if (L.total < 120u * 1024u) L.total = 120u * 1024u;
    return L;
}
}  // namespace


// Bounded wait used only while draining (ignores the abort flag).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity, int* status) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > ICA_WAIT_NS) {
            atomicOr(status, DEV_TIMEOUT);
            return;
        }
    }
}

__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Restart tile -> MMA A operands, by the kEpiWarps epilogue warps (warp index w = 2..).
// hi = bf16(b) goes to shared memory (K-major, 128-byte swizzle, K-block kb of 64 columns at
// kb * 16 KB); with the split, lo = bf16(b - hi) goes beside it (second half of the A region,
// smem_lo) or to tensor memory (lo_tmem != 0: lane = row, K step ks at 8 columns from
// lo_tmem + 8 ks; each warp writes its own lane quarter, as tcgen05.st requires). Rows at or
// beyond M_act are zero. Row m of the tile is restart act[m0 + m] (or m0 + m when act is null).
// ldcg: read B through L2 (rows written by other CTAs of a persistent launch).
// with_lo = false: the low term is not written (iterations that use the high term alone).
template <bool SPLIT, bool LO_TMEM>
__device__ __forceinline__ void convert_restart_tile(const float* __restrict__ B32, int ldb, const int* act, int m0,
                                                     int M_act, int n_pad, uint32_t sA, uint32_t a_bytes,
                                                     uint32_t lo_tmem, bool ldcg, bool with_lo = true) {
    auto lo_of = [](uint32_t hp, float x, float y) {
        return pack_bf16x2(x - __uint_as_float(hp << 16), y - __uint_as_float(hp & 0xFFFF0000u));
    };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (LO_TMEM) {
        // warp (lane quarter q, group h) takes row 32 q + lane and K steps h, h + 4, ...
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int row = q * 32 + lane, gm = m0 + row;
        const bool live = gm < M_act;
        const int r = live ? (act ? (ldcg ? __ldcg(act + gm) : act[gm]) : gm) : 0;
        const float* src = B32 + static_cast<int64_t>(r) * ldb;
        const int ksteps = n_pad / 16;
        for (int ks = h; ks < ksteps; ks += kEpiWarps / 4) {
            float4 v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (live) {
                    const float4* p = reinterpret_cast<const float4*>(src + ks * 16) + i;
                    v[i] = ldcg ? __ldcg(p) : *p;
                }
            }
            uint32_t hp[8], lp[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                hp[2 * i] = pack_bf16x2(v[i].x, v[i].y);
                hp[2 * i + 1] = pack_bf16x2(v[i].z, v[i].w);
                lp[2 * i] = lo_of(hp[2 * i], v[i].x, v[i].y);
                lp[2 * i + 1] = lo_of(hp[2 * i + 1], v[i].z, v[i].w);
            }
#pragma unroll
            for (int half = 0; half < 2; ++half) {  // the two 8-element chunks of the K step
                const int ch = ks * 2 + half;
                const uint32_t addr = sA + static_cast<uint32_t>(ch >> 3) * 16384u + sw128_off(row, ch & 7);
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(hp[4 * half]),
                             "r"(hp[4 * half + 1]), "r"(hp[4 * half + 2]), "r"(hp[4 * half + 3])
                             : "memory");
            }
            if (with_lo) tmem_st8(lo_tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(ks * 8), lp);
        }
        tmem_st_wait();
    } else {
        const int et = threadIdx.x - 64;
        const int cpr = n_pad / 8;
        for (int idx = et; idx < kTcRows * cpr; idx += 32 * kEpiWarps) {
            const int row = idx / cpr, ch = idx % cpr;
            const int gm = m0 + row;
            float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
            if (gm < M_act) {
                const int r = act ? (ldcg ? __ldcg(act + gm) : act[gm]) : gm;
                const float4* src = reinterpret_cast<const float4*>(B32 + static_cast<int64_t>(r) * ldb + ch * 8);
                v0 = ldcg ? __ldcg(src) : src[0];
                v1 = ldcg ? __ldcg(src + 1) : src[1];
            }
            const uint32_t addr = sA + static_cast<uint32_t>(ch >> 3) * 16384u + sw128_off(row, ch & 7);
            const uint32_t h0 = pack_bf16x2(v0.x, v0.y), h1 = pack_bf16x2(v0.z, v0.w), h2 = pack_bf16x2(v1.x, v1.y),
                           h3 = pack_bf16x2(v1.z, v1.w);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(h0), "r"(h1), "r"(h2), "r"(h3)
                         : "memory");
            if (SPLIT && with_lo) {  // residuals b - float(bf16(b)) in the second half
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr + (a_bytes >> 1)),
                             "r"(lo_of(h0, v0.x, v0.y)), "r"(lo_of(h1, v0.z, v0.w)), "r"(lo_of(h2, v1.x, v1.y)),
                             "r"(lo_of(h3, v1.z, v1.w))
                             : "memory");
            }
        }
    }
    fence_proxy_async_smem();
}

// Restart tile -> E4M3 A operands of the FP8 first product, by the kEpiWarps epilogue warps: with
// x = b[r][k] * colscale[k], hi = e4m3(x) and lo = e4m3(x - hi) (together about 8 significant
// bits, where one E4M3 term carries 4), each K-major with 128-byte swizzle, K block kb of 128
// entries at kb * 16 KB; lo at byte offset lo_off. Zero for k >= n and for rows at or beyond
// M_act; r = act[m0 + m]; k < n8. B32 rows hold ldb = round_up(n, 16) entries, zero from n on (the
// padding of the reduced dimension). |x| <= 256, so neither term saturates.
__device__ __forceinline__ void convert_restart_tile_e4m3(const float* __restrict__ B32, int ldb, const int* act,
                                                          int m0, int M_act, int n, int n8, uint32_t sA,
                                                          uint32_t lo_off, const float* __restrict__ colscale) {
    const int et = threadIdx.x - 64;
    const int cpr = n8 / 16;  // 16-entry (16-byte) chunks per row
    for (int idx = et; idx < kTcRows * cpr; idx += 32 * kEpiWarps) {
        const int row = idx / cpr, ch = idx % cpr;
        const int gm = m0 + row;
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
        if (gm < M_act && ch * 16 < n) {  // entries n..ldb-1 of a row are zero; ldb is a multiple of 16
            const int r = __ldcg(act + gm);
            const float4* src = reinterpret_cast<const float4*>(B32 + static_cast<int64_t>(r) * ldb + ch * 16);
            const float4* cs = reinterpret_cast<const float4*>(colscale + ch * 16);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 x = __ldcg(src + i), c = __ldg(cs + i);
                v[4 * i] = x.x * c.x;
                v[4 * i + 1] = x.y * c.y;
                v[4 * i + 2] = x.z * c.z;
                v[4 * i + 3] = x.w * c.w;
            }
        }
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            hw[i] = pack_e4m3x4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            const float2 h01 = e4m3x2_to_float2(hw[i] & 0xffffu), h23 = e4m3x2_to_float2(hw[i] >> 16);
            lw[i] = pack_e4m3x4(v[4 * i] - h01.x, v[4 * i + 1] - h01.y, v[4 * i + 2] - h23.x, v[4 * i + 3] - h23.y);
        }
        const uint32_t addr = sA + static_cast<uint32_t>(ch >> 3) * 16384u + sw128_off(row, ch & 7);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(hw[0]), "r"(hw[1]), "r"(hw[2]),
                     "r"(hw[3])
                     : "memory");
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr + lo_off), "r"(lw[0]), "r"(lw[1]),
                     "r"(lw[2]), "r"(lw[3])
                     : "memory");
    }
    fence_proxy_async_smem();
}

}  // namespace ica
