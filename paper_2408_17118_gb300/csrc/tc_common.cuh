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
// Restart rows as two BF16 terms (hi = bf16(b), lo = bf16(b - hi)) in the first product, for the
// 192-sample chunks (n_pad <= 64): Z = B_hi X~ + B_lo X~ carries b to about 16 bits instead of 8,
// so that the BF16 stage's step distance can fall below its tolerance instead of stalling at the
// rounding noise of b. Costs one more MMA per K step of the first product.
#ifndef ICA_TC_SPLIT_B
#define ICA_TC_SPLIT_B 1
#endif
__host__ __device__ constexpr bool tc_split_b(int TC) { return ICA_TC_SPLIT_B && TC == 192; }
// Second products issued by two threads (on different schedulers) into two accumulators, summed
// when read out: measured on GB300, one thread sustained one M128 K16 MMA per 67 cycles at
// N <= 64 and two threads one per 50 (N = 64) or 41 (N = 16) cycles. Both accumulators fit TMEM
// next to the Z buffers for TC = 192 (n_pad <= 64) and TC = 128 (n_pad <= 128).
__host__ __device__ constexpr int tc_g2_issuers(int TC) { return TC == 64 ? 1 : 2; }
__host__ __device__ constexpr uint32_t tc_d2_cols(int TC) { return TC == 192 ? 64u : (TC == 128 ? 128u : 256u); }

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
    uint32_t a_bytes, xsub_bytes, xn_bytes, xstage_bytes, p_bytes, stages, off_x, off_p, off_bar, total;
};
// reserve: bytes of the 227 KB per-CTA shared memory left for the kernel's static shared memory
TcLayout tc_layout(int n_pad, bool moments_only, int TC, int NB, bool KT, uint32_t reserve = 0) {
    TcLayout L{};
    L.a_bytes = static_cast<uint32_t>((n_pad + 63) / 64) * 16384u * (tc_split_b(TC) ? 2u : 1u);
    L.xsub_bytes = static_cast<uint32_t>(n_pad) * 128u;
    L.xn_bytes = static_cast<uint32_t>(TC / 64) * L.xsub_bytes;  // X~ tile: n_pad rows x TC samples
    // + X~^T tile: ceil(n_pad / 64) K-blocks of TC rows x 128 bytes
    L.xstage_bytes = L.xn_bytes + (KT ? static_cast<uint32_t>((n_pad + 63) / 64) * static_cast<uint32_t>(TC) * 128u : 0u);
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

}  // namespace ica
