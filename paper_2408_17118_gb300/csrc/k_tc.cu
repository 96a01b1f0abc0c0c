// Fused tcgen05 iteration of the matrix form (Section 3.1; the update of Algorithm 2) for a
// tile of 128 active restarts and a contiguous range of samples:
//
//   for each chunk of TC samples:   Z    = B_tile X~_chunk          (tcgen05, D1 in TMEM)
//                                   P    = bf16(Z o Z o Z)          (registers -> swizzled SMEM)
//                                   Acc += P X~_chunk^T             (tcgen05, D2 in TMEM)
//
// Z exists only in TMEM and registers: it never reaches device memory. The same TMA-loaded
// X~ chunk (n_pad rows x TC samples, 128-byte swizzle) is the MN-major B operand of the first
// product (contraction over the reduced dimension) and the K-major B operand of the second
// (contraction over samples). The epilogue also accumulates sum z^2 and sum z^4 per restart
// (and sum (z^2 - 1)^2 in the moments-only variant, which skips the second product and is
// used for the kurtosis of candidates, Eq. 2).
//
// Warp roles (320 threads): warp 0 issues TMA loads, warp 1 allocates TMEM and issues MMAs
// (one thread), warps 2..9 convert TMEM rows (warp w reads TMEM lanes 32*(w%4).., half
// (w-2)/4 of the chunk's columns). Every wait is bounded (ICA_WAIT_NS): on timeout the CTA
// raises the device status word, drains its outstanding copies and MMAs, frees TMEM and
// returns.
#include "common.cuh"
#include "internal.h"

namespace ica {

int tc_chunk(int n_pad) { return n_pad <= 128 ? 128 : 64; }

namespace {
constexpr int kBars = 40;
struct TcLayout {
    uint32_t a_bytes, xsub_bytes, xstage_bytes, p_bytes, stages, off_x, off_p, off_bar, total;
};
TcLayout tc_layout(int n_pad, bool moments_only, int TC) {
    TcLayout L{};
    L.a_bytes = static_cast<uint32_t>((n_pad + 63) / 64) * 16384u;
    L.xsub_bytes = static_cast<uint32_t>(n_pad) * 128u;
    L.xstage_bytes = static_cast<uint32_t>(TC / 64) * L.xsub_bytes;
    L.p_bytes = moments_only ? 0u : static_cast<uint32_t>(TC / 64) * 16384u;
    const uint32_t fixed = L.a_bytes + 2u * L.p_bytes + 4096u + 1024u;  // + barriers/scratch + alignment
    const uint32_t budget = 227u * 1024u;
    uint32_t st = (budget - fixed) / L.xstage_bytes;
    if (st > 8) st = 8;
    L.stages = st;
    L.off_x = L.a_bytes;
    L.off_p = L.off_x + st * L.xstage_bytes;
    L.off_bar = L.off_p + 2u * L.p_bytes;
    L.total = L.off_bar + 4096u + 1024u;
    // one CTA per SM: the kernel allocates all 512 TMEM columns
    if (L.total < 120u * 1024u) L.total = 120u * 1024u;
    return L;
}
}  // namespace

size_t tc_smem_bytes(int n_pad, bool moments_only, int* stages_out) {
    const TcLayout L = tc_layout(n_pad, moments_only, tc_chunk(n_pad));
    if (stages_out) *stages_out = static_cast<int>(L.stages);
    return L.total;
}

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

template <int TC, bool MOMENTS_ONLY>
__global__ void __launch_bounds__(320, 1)
    fused_tc_kernel(const __grid_constant__ CUtensorMap xmap, const float* __restrict__ B32, int ldb,
                    const int* __restrict__ act_idx, int M_act, int n_pad, int64_t T, int chunks_per_split,
                    int total_chunks, int stages, uint32_t a_bytes, uint32_t xsub_bytes, uint32_t off_x,
                    uint32_t off_p, uint32_t off_bar, float* __restrict__ part_acc, float* __restrict__ part_mom,
                    int part_rows, int* status) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    const uint32_t base_u32 = (raw_u32 + 1023u) & ~1023u;
    uint8_t* base = smem_raw + (base_u32 - raw_u32);
    const uint32_t xstage_bytes = static_cast<uint32_t>(TC / 64) * xsub_bytes;
    constexpr uint32_t p_bytes = static_cast<uint32_t>(TC / 64) * 16384u;
    const uint32_t sA = base_u32, sX = base_u32 + off_x, sP = base_u32 + off_p;
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + off_bar);
    uint64_t* full = bars;          // [8]  X~ stage loaded
    uint64_t* empty = bars + 8;     // [8]  X~ stage released by the MMAs that read it
    uint64_t* d1_full = bars + 16;  // [2]  Z chunk ready in TMEM
    uint64_t* d1_empty = bars + 18; // [2]  Z chunk read out by the 8 epilogue warps
    uint64_t* p_full = bars + 20;   // [2]  P chunk written to SMEM by the 8 epilogue warps
    uint64_t* p_empty = bars + 22;  // [2]  P chunk consumed by the second product
    uint64_t* d2_full = bars + 24;  //      accumulator complete
    uint64_t* mma_done = bars + 25; //      every MMA of this CTA retired (teardown)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kBars);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* mom_sm = reinterpret_cast<float*>(bars + kBars + 2);  // [128][4]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = blockIdx.x, tile = blockIdx.y;
    const int m0 = tile * kTcRows;
    const int c_begin = split * chunks_per_split;
    const int c_end = min(total_chunks, c_begin + chunks_per_split);
    const int nch = c_end - c_begin;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&d1_full[b], 1);
            mbar_init(&d1_empty[b], 8);
            mbar_init(&p_full[b], 8);
            mbar_init(&p_empty[b], 1);
        }
        mbar_init(d2_full, 1);
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) tma_prefetch_desc(&xmap);
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    if (warp >= 2) {
        // restart tile -> BF16, K-major, 128-byte swizzle: K-block kb (64 columns) at kb*16 KB
        const int et = threadIdx.x - 64;
        const int cpr = n_pad / 8;
        for (int idx = et; idx < kTcRows * cpr; idx += 256) {
            const int row = idx / cpr, ch = idx % cpr;
            const int gm = m0 + row;
            float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
            if (gm < M_act) {
                const int r = act_idx ? act_idx[gm] : gm;
                const float4* src = reinterpret_cast<const float4*>(B32 + static_cast<int64_t>(r) * ldb + ch * 8);
                v0 = src[0];
                v1 = src[1];
            }
            const uint32_t addr = sA + static_cast<uint32_t>(ch >> 3) * 16384u + sw128_off(row, ch & 7);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(pack_bf16x2(v0.x, v0.y)),
                         "r"(pack_bf16x2(v0.z, v0.w)), "r"(pack_bf16x2(v1.x, v1.y)), "r"(pack_bf16x2(v1.z, v1.w))
                         : "memory");
        }
        fence_proxy_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tD2 = tmem;
    const uint32_t tD1_0 = tmem + 256u, tD1_1 = tmem + 256u + static_cast<uint32_t>(TC);

    if (warp == 0) {
        // ------------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int issued = 0;
            for (int c = 0; c < nch; ++c) {
                const int s = c % stages;
                if (c >= stages && !mbar_wait(&empty[s], static_cast<uint32_t>((c / stages) - 1) & 1u, abort_flag,
                                              status))
                    break;
                mbar_arrive_expect_tx(&full[s], xstage_bytes);
                const int tg = (c_begin + c) * TC;
#pragma unroll
                for (int sub = 0; sub < TC / 64; ++sub)
                    tma_load_2d(sX + static_cast<uint32_t>(s) * xstage_bytes + static_cast<uint32_t>(sub) * xsub_bytes,
                                &xmap, &full[s], tg + sub * 64, 0);
                ++issued;
            }
            // drain: every issued load must land before the CTA can exit
            for (int s = 0; s < stages && s < issued; ++s) {
                const int c_last = s + ((issued - 1 - s) / stages) * stages;
                mbar_drain(&full[s], static_cast<uint32_t>(c_last / stages) & 1u, status);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t id1 = idesc_bf16(128, TC, 1);  // B operand MN-major (samples contiguous)
            const uint32_t id2 = idesc_bf16(128, static_cast<uint32_t>(n_pad), 0);
            bool ok = true;
            for (int c = 0; c <= nch && ok; ++c) {
                if (c < nch) {
                    const int s = c % stages, b = c & 1;
                    ok = mbar_wait(&full[s], static_cast<uint32_t>(c / stages) & 1u, abort_flag, status);
                    if (ok && c >= 2) ok = mbar_wait(&d1_empty[b], static_cast<uint32_t>((c - 2) >> 1) & 1u, abort_flag, status);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t xs = sX + static_cast<uint32_t>(s) * xstage_bytes;
                    const uint32_t d1 = b ? tD1_1 : tD1_0;
                    for (int ks = 0; ks < n_pad / 16; ++ks) {
                        const uint64_t ad = sw128_desc(sA + static_cast<uint32_t>(ks >> 2) * 16384u +
                                                           static_cast<uint32_t>(ks & 3) * 32u,
                                                       16u, 1024u);
                        const uint64_t bd = sw128_desc(xs + static_cast<uint32_t>(ks) * 2048u, xsub_bytes, 1024u);
                        umma_bf16(d1, ad, bd, id1, ks > 0 ? 1u : 0u);
                    }
                    umma_commit(&d1_full[b]);
                    if (MOMENTS_ONLY) umma_commit(&empty[s]);
                }
                if (!MOMENTS_ONLY && c >= 1) {
                    const int cp = c - 1, sp = cp % stages, bp = cp & 1;
                    ok = mbar_wait(&p_full[bp], static_cast<uint32_t>(cp >> 1) & 1u, abort_flag, status);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t xs = sX + static_cast<uint32_t>(sp) * xstage_bytes;
                    const uint32_t ps = sP + static_cast<uint32_t>(bp) * p_bytes;
#pragma unroll
                    for (int ks = 0; ks < TC / 16; ++ks) {
                        const uint64_t ad = sw128_desc(ps + static_cast<uint32_t>(ks >> 2) * 16384u +
                                                           static_cast<uint32_t>(ks & 3) * 32u,
                                                       16u, 1024u);
                        const uint64_t bd = sw128_desc(xs + static_cast<uint32_t>(ks >> 2) * xsub_bytes +
                                                           static_cast<uint32_t>(ks & 3) * 32u,
                                                       16u, 1024u);
                        umma_bf16(tD2, ad, bd, id2, (cp > 0 || ks > 0) ? 1u : 0u);
                    }
                    umma_commit(&p_empty[bp]);
                    umma_commit(&empty[sp]);
                }
            }
            if (!MOMENTS_ONLY) umma_commit(d2_full);
            umma_commit(mma_done);
            mbar_drain(mma_done, 0u, status);
        }
    } else {
        // ------------------------------------------------------------------ epilogue warps
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
        constexpr int CW = TC / 2;
        float2 s2 = make_float2(0.f, 0.f), s4 = make_float2(0.f, 0.f);
        float sq = 0.f;
        bool ok = true;
        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            ok = __all_sync(0xffffffffu, mbar_wait(&d1_full[b], static_cast<uint32_t>(c >> 1) & 1u, abort_flag, status));
            if (!ok) break;
            tc_fence_after();
            float v[CW];
            const uint32_t d1 = (b ? tD1_1 : tD1_0) + lane_off + static_cast<uint32_t>(h * CW);
#pragma unroll
            for (int g = 0; g < CW / 32; ++g) tmem_ld32(d1 + static_cast<uint32_t>(g * 32), *reinterpret_cast<float(*)[32]>(&v[g * 32]));
            tmem_ld_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&d1_empty[b]);
            uint32_t pk[CW / 2];
            const int64_t tbase = static_cast<int64_t>(c_begin + c) * TC + h * CW;
#pragma unroll
            for (int i = 0; i < CW; i += 2) {
                const float2 z = make_float2(v[i], v[i + 1]);
                const float2 z2 = mul2(z, z);
                s2 = add2(s2, z2);
                s4 = fma2(z2, z2, s4);
                if (MOMENTS_ONLY) {
                    const float e0 = (tbase + i < T) ? z2.x - 1.f : 0.f;
                    const float e1 = (tbase + i + 1 < T) ? z2.y - 1.f : 0.f;
                    sq = fmaf(e0, e0, fmaf(e1, e1, sq));
                } else {
                    const float2 z3 = mul2(z2, z);
                    pk[i / 2] = pack_bf16x2(z3.x, z3.y);
                }
            }
            if (!MOMENTS_ONLY) {
                if (c >= 2) {
                    ok = __all_sync(0xffffffffu,
                                    mbar_wait(&p_empty[b], static_cast<uint32_t>((c - 2) >> 1) & 1u, abort_flag, status));
                    if (!ok) break;
                }
                const uint32_t pbase = sP + static_cast<uint32_t>(b) * p_bytes;
#pragma unroll
                for (int g = 0; g < CW / 8; ++g) {
                    const int col = h * CW + g * 8;  // sample within the chunk
                    const uint32_t addr = pbase + static_cast<uint32_t>(col >> 6) * 16384u +
                                          sw128_off(static_cast<uint32_t>(row), static_cast<uint32_t>((col & 63) >> 3));
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(pk[g * 4 + 0]),
                                 "r"(pk[g * 4 + 1]), "r"(pk[g * 4 + 2]), "r"(pk[g * 4 + 3])
                                 : "memory");
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&p_full[b]);
            }
        }
        const int grow = m0 + row;
        const int64_t prow = static_cast<int64_t>(split) * part_rows + grow;
        if (!MOMENTS_ONLY && ok) {
            ok = __all_sync(0xffffffffu, mbar_wait(d2_full, 0u, abort_flag, status));
            if (ok) {
                tc_fence_after();
                const int half = n_pad / 2;
                for (int g = 0; g < half / 8; ++g) {
                    const int col = h * half + g * 8;
                    float v8[8];
                    tmem_ld8(tD2 + lane_off + static_cast<uint32_t>(col), v8);
                    tmem_ld_wait();
                    if (grow < M_act) {
                        float4* dst = reinterpret_cast<float4*>(part_acc + prow * n_pad + col);
                        dst[0] = make_float4(v8[0], v8[1], v8[2], v8[3]);
                        dst[1] = make_float4(v8[4], v8[5], v8[6], v8[7]);
                    }
                }
            }
        }
        if (h == 1) {
            mom_sm[row * 4 + 0] = s2.x + s2.y;
            mom_sm[row * 4 + 1] = s4.x + s4.y;
            mom_sm[row * 4 + 2] = sq;
        }
        named_bar_sync(1, 256);
        if (h == 0 && grow < M_act) {
            part_mom[prow * 4 + 0] = s2.x + s2.y + mom_sm[row * 4 + 0];
            part_mom[prow * 4 + 1] = s4.x + s4.y + mom_sm[row * 4 + 1];
            part_mom[prow * 4 + 2] = sq + mom_sm[row * 4 + 2];
            part_mom[prow * 4 + 3] = 0.f;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

template <int TC, bool MO>
static cudaError_t launch_tc_impl(cudaStream_t s, const CUtensorMap& xmap, const float* B32, int ldb,
                                  const int* act_idx, int M_act, int n_pad, int64_t T, int splits,
                                  int chunks_per_split, int total_chunks, float* part_acc, float* part_mom,
                                  int part_rows, int* status) {
    const TcLayout L = tc_layout(n_pad, MO, TC);
    cudaError_t e = cudaFuncSetAttribute(fused_tc_kernel<TC, MO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L.total));
    if (e != cudaSuccess) return e;
    const dim3 grid(splits, (M_act + kTcRows - 1) / kTcRows);
    fused_tc_kernel<TC, MO><<<grid, 320, L.total, s>>>(xmap, B32, ldb, act_idx, M_act, n_pad, T, chunks_per_split,
                                                       total_chunks, static_cast<int>(L.stages), L.a_bytes,
                                                       L.xsub_bytes, L.off_x, L.off_p, L.off_bar, part_acc, part_mom,
                                                       part_rows, status);
    return cudaGetLastError();
}

cudaError_t launch_fused_tc(cudaStream_t s, bool moments_only, const CUtensorMap& xmap, const float* B32, int ldb,
                            const int* act_idx, int M_act, int n_pad, int64_t T, int splits, int chunks_per_split,
                            int total_chunks, float* part_acc, float* part_mom, int part_rows, int* status) {
    const int TC = tc_chunk(n_pad);
    if (TC == 128) {
        return moments_only ? launch_tc_impl<128, true>(s, xmap, B32, ldb, act_idx, M_act, n_pad, T, splits,
                                                        chunks_per_split, total_chunks, part_acc, part_mom,
                                                        part_rows, status)
                            : launch_tc_impl<128, false>(s, xmap, B32, ldb, act_idx, M_act, n_pad, T, splits,
                                                         chunks_per_split, total_chunks, part_acc, part_mom,
                                                         part_rows, status);
    }
    return moments_only ? launch_tc_impl<64, true>(s, xmap, B32, ldb, act_idx, M_act, n_pad, T, splits,
                                                   chunks_per_split, total_chunks, part_acc, part_mom, part_rows,
                                                   status)
                        : launch_tc_impl<64, false>(s, xmap, B32, ldb, act_idx, M_act, n_pad, T, splits,
                                                    chunks_per_split, total_chunks, part_acc, part_mom, part_rows,
                                                    status);
}

}  // namespace ica
