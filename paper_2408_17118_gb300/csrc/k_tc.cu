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
// used for the kurtosis of candidates, Eq. 2); the update variant accumulates the moments
// only when asked (the first iterations, whose kurtosis trajectory is kept per restart).
//
// Warp roles (640 threads): warp 0 issues TMA loads; warp 1 allocates TMEM and issues the first
// products (one thread); warps 18 and 19 issue the second products (one thread each: even and
// odd K steps into two accumulators when TMEM has room, tc_g2_issuers); warps 2..17 convert
// TMEM rows (warp w reads TMEM lanes 32*(w%4).., quarter (w-2)/4 of the chunk's columns). The
// issuing threads sit on different schedulers: measured on GB300, one thread issuing both
// products spent about 100 cycles per tcgen05.mma while sharing its scheduler with four busy
// epilogue warps, and splitting the issue cut the time of a 64 x 1024 x 2e6 step by a quarter.
// Every wait is bounded (ICA_WAIT_NS): on timeout the CTA raises the device status word, drains
// its outstanding copies and MMAs, frees TMEM and returns.
#include "tc_common.cuh"

namespace ica {

int tc_chunk(int n_pad) { return n_pad <= 64 ? ICA_TC_SMALL_CHUNK : (n_pad <= 128 ? 128 : 64); }
int tc_buffers(int n_pad) { return n_pad <= 64 ? ICA_TC_SMALL_NB : 2; }
size_t tc_smem_bytes(int n_pad, bool moments_only, int* stages_out) {
    const TcLayout L = tc_layout(n_pad, moments_only, tc_chunk(n_pad), tc_buffers(n_pad));
    if (stages_out) *stages_out = static_cast<int>(L.stages);
    return L.total;
}

template <int TC, int NB, bool MOMENTS_ONLY, bool MOMENTS>
__global__ void __launch_bounds__(kThreads, 1)
    fused_tc_kernel(const __grid_constant__ CUtensorMap xmap, const float* __restrict__ B32, int ldb,
                    const int* __restrict__ act_idx, const int* __restrict__ count_dev, int M_act_host, int n_pad, int64_t T, int chunks_per_split,
                    int total_chunks, int stages, uint32_t a_bytes, uint32_t xsub_bytes, uint32_t xstage_bytes,
                    uint32_t off_x,
                    uint32_t off_p, uint32_t off_bar, float* __restrict__ part_acc, float* __restrict__ part_mom,
                    int part_rows, int* status, int shape_ctas, int* shape_out, int use_lo) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    const uint32_t base_u32 = (raw_u32 + 1023u) & ~1023u;
    uint8_t* base = smem_raw + (base_u32 - raw_u32);
    constexpr uint32_t p_bytes = static_cast<uint32_t>(TC / 64) * 16384u;
    const uint32_t sA = base_u32, sX = base_u32 + off_x, sP = base_u32 + off_p;
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + off_bar);
    uint64_t* full = bars;          // [8]  X~ stage loaded
    uint64_t* empty = bars + 8;     // [8]  X~ stage released by the MMAs that read it
    uint64_t* d1_full = bars + 16;  // [NB] Z chunk ready in TMEM
    uint64_t* d1_empty = bars + 19; // [NB] Z chunk read out by the 16 epilogue warps
    uint64_t* p_full = bars + 22;   // [NB] P chunk written to SMEM by the 16 epilogue warps
    uint64_t* d2_full = bars + 28;  //      accumulator complete
    uint64_t* mma_done = bars + 29; //      every MMA of this CTA retired (teardown)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kBars);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* mom_sm = reinterpret_cast<float*>(bars + kBars + 2);  // [3][128][4]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    pdl_wait();  // the previous grid (finalize of the last update) wrote B, the list and the count
    pdl_trigger();
    const int M_act = count_dev ? *count_dev : M_act_host;
    int split = blockIdx.x, tile = blockIdx.y, cps = chunks_per_split;
    if (shape_ctas > 0) {
        // launch shape from the device count (the host knows only an upper bound): tiles of 128
        // active rows x splits of the sample range, at most one wave (tc_device_shape)
        int tiles, sp;
        tc_device_shape(M_act, shape_ctas, total_chunks, &tiles, &sp, &cps);
        const int b = blockIdx.x;
        if (b == 0 && threadIdx.x == 0 && shape_out) {
            shape_out[0] = sp;
            shape_out[1] = tiles * kTcRows;
        }
        if (b >= tiles * sp) return;
        tile = b / sp;
        split = b % sp;
        part_rows = tiles * kTcRows;
    }
    const int m0 = tile * kTcRows;
    if (m0 >= M_act) return;  // grid sized for an upper bound of the active count
    const int c_begin = split * cps;
    const int c_end = min(total_chunks, c_begin + cps);
    const int nch = c_end - c_begin;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], MOMENTS_ONLY ? 1 : tc_g2_issuers(TC));  // every second-product issuer
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(&d1_full[b], 1);
            mbar_init(&d1_empty[b], kEpiWarps);
            mbar_init(&p_full[b], kEpiWarps);
        }
        mbar_init(d2_full, tc_g2_issuers(TC));
        mbar_init(mma_done, MOMENTS_ONLY ? 1 : 1 + tc_g2_issuers(TC));  // one commit per MMA-issuing thread
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) tma_prefetch_desc(&xmap);
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    constexpr bool kSplit = tc_split_b(TC), kLoTmem = tc_lo_in_tmem(TC);
    if (!kLoTmem && warp >= 2 && warp < 2 + kEpiWarps)  // restart tile -> BF16 hi (+ lo) in shared memory
        convert_restart_tile<kSplit, false>(B32, ldb, act_idx, m0, M_act, n_pad, sA, a_bytes, 0u, false, use_lo != 0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tD2 = tmem;
    constexpr int G2S = tc_g2_issuers(TC);
    constexpr uint32_t kD2Cols = tc_d2_cols(TC);
    constexpr uint32_t kD1Col = G2S * kD2Cols;  // Z buffers after the G2S accumulators
    static_assert(kD1Col + NB * TC <= 512, "D2 and the Z buffers must fit in 512 TMEM columns");
    static_assert(NB >= 2 && NB <= 3, "barrier slots exist for up to three Z / P buffers");
    constexpr uint32_t kALoCol = tc_alo_col(TC, NB);  // B's low term (kLoTmem): n_pad / 2 columns
    static_assert(!kLoTmem || kALoCol + (TC == 128 ? 64u : 128u) <= 512, "B's low term must fit TMEM");
    if constexpr (kLoTmem) {
        // the low term goes to tensor memory, whose address is known only now: the epilogue warps
        // convert the tile, then meet the first-product issuer (warp 1) at a named barrier
        if (warp >= 2 && warp < 2 + kEpiWarps) {
            convert_restart_tile<kSplit, true>(B32, ldb, act_idx, m0, M_act, n_pad, sA, a_bytes, tmem + kALoCol,
                                               false, use_lo != 0);
            tc_fence_before();
        }
        if (warp >= 1 && warp < 2 + kEpiWarps) named_bar_sync(10, 32 * (1 + kEpiWarps));
        if (warp == 1) tc_fence_after();
    }

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
                const uint32_t stage = sX + static_cast<uint32_t>(s) * xstage_bytes;
#pragma unroll
                for (int sub = 0; sub < TC / 64; ++sub)
                    tma_load_2d(stage + static_cast<uint32_t>(sub) * xsub_bytes, &xmap, &full[s], tg + sub * 64, 0);
                ++issued;
            }
            // drain: every issued load must land before the CTA can exit
            for (int s = 0; s < stages && s < issued; ++s) {
                const int c_last = s + ((issued - 1 - s) / stages) * stages;
                mbar_drain(&full[s], static_cast<uint32_t>(c_last / stages) & 1u, status);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------------ first-product issuer
        if (lane == 0) {
            constexpr uint32_t id1 = idesc_bf16(128, TC, 1u);  // B: X~ MN-major
            // Descriptors are built once; a K step only moves the start-address field (address >> 4,
            // bits 0-13), which cannot carry into the next field for shared addresses below 256 KB.
            const uint64_t a1_desc = sw128_desc(sA, 16u, 1024u);
            const uint64_t b1_desc = sw128_desc(sX, xsub_bytes, 1024u);
            const uint32_t stage16 = xstage_bytes >> 4;
            const int ksteps1 = n_pad / 16;
            bool ok = true;
            for (int c = 0; c < nch && ok; ++c) {
                const int s = c % stages, b = c % NB;
                ok = mbar_wait(&full[s], static_cast<uint32_t>(c / stages) & 1u, abort_flag, status);
                if (ok && c >= NB)
                    ok = mbar_wait(&d1_empty[b], static_cast<uint32_t>((c - NB) / NB) & 1u, abort_flag, status);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d1 = tmem + kD1Col + static_cast<uint32_t>(b * TC);
                const uint64_t b1s = b1_desc + static_cast<uint64_t>(static_cast<uint32_t>(s) * stage16);
#pragma unroll
                for (int ks = 0; ks < 16; ++ks) {
                    if (ks >= ksteps1) break;
                    const uint32_t a_off = ((ks >> 2) * 16384u + (ks & 3) * 32u) >> 4;
                    const uint32_t b_off = (static_cast<uint32_t>(ks) * 2048u) >> 4;
                    umma_bf16(d1, a1_desc + a_off, b1s + b_off, id1, ks > 0 ? 1u : 0u);
                }
                if (!use_lo) {
                } else if constexpr (kLoTmem) {
#pragma unroll
                    for (int ks = 0; ks < 16; ++ks) {
                        if (ks >= ksteps1) break;
                        const uint32_t b_off = (static_cast<uint32_t>(ks) * 2048u) >> 4;
                        umma_bf16_tmem_a_acc(d1, tmem + kALoCol + static_cast<uint32_t>(ks) * 8u, b1s + b_off, id1);
                    }
                } else if constexpr (kSplit) {
                    const uint64_t a1_lo = a1_desc + static_cast<uint64_t>((a_bytes >> 1) >> 4);
#pragma unroll
                    for (int ks = 0; ks < 16; ++ks) {
                        if (ks >= ksteps1) break;
                        const uint32_t a_off = ((ks >> 2) * 16384u + (ks & 3) * 32u) >> 4;
                        const uint32_t b_off = (static_cast<uint32_t>(ks) * 2048u) >> 4;
                        umma_bf16_acc(d1, a1_lo + a_off, b1s + b_off, id1);
                    }
                }
                umma_commit(&d1_full[b]);
                if (MOMENTS_ONLY) umma_commit(&empty[s]);  // no second product reads the stage
            }
            umma_commit(mma_done);
            mbar_drain(mma_done, 0u, status);
        }
    } else if (warp == kG2Warp || warp == kG2bWarp) {
        // ------------------------------------------------------------------ second-product issuers
        // Threads of their own (on other schedulers than the first-product issuer), so that the
        // instruction streams overlap; the products write different TMEM columns and every
        // shared operand they share is ordered by the barriers (P(c) exists only after the
        // first product of chunk c retired and the epilogue consumed it). Issuer gi of G2S takes
        // the K steps j = gi mod G2S into accumulator gi.
        const int gi = warp - kG2Warp;
        if (!MOMENTS_ONLY && lane == 0 && gi < G2S) {
            const uint32_t id2 = idesc_bf16(128, static_cast<uint32_t>(n_pad), 0);
            const uint32_t dacc = tD2 + static_cast<uint32_t>(gi) * kD2Cols;
            // Per-K-step descriptors of stage 0 / buffer 0, built once: inside the chunk loop an MMA
            // costs two 64-bit adds (stage and buffer offsets) besides the instruction itself.
            constexpr int KSI = TC / 16 / G2S;  // K steps of this issuer: gi, gi + G2S, ...
            uint64_t pd[KSI], xd[KSI];
#pragma unroll
            for (int j = 0; j < KSI; ++j) {
                const uint32_t ks = static_cast<uint32_t>(gi + j * G2S);
                pd[j] = sw128_desc(sP + (ks >> 2) * 16384u + (ks & 3u) * 32u, 16u, 1024u);
                xd[j] = sw128_desc(sX + (ks >> 2) * xsub_bytes + (ks & 3u) * 32u, 16u, 1024u);
            }
            const uint32_t stage16 = xstage_bytes >> 4;
            bool ok = true;
            int s = 0, b = 0;
            uint32_t par = 0u;
            for (int c = 0; c < nch && ok; ++c) {
                ok = mbar_wait(&p_full[b], par, abort_flag, status);
                if (!ok) break;
                tc_fence_after();
                const uint64_t po = static_cast<uint64_t>((static_cast<uint32_t>(b) * p_bytes) >> 4);
                const uint64_t xo = static_cast<uint64_t>(static_cast<uint32_t>(s) * stage16);
                umma_bf16(dacc, pd[0] + po, xd[0] + xo, id2, c > 0 ? 1u : 0u);
#pragma unroll
                for (int j = 1; j < KSI; ++j) umma_bf16_acc(dacc, pd[j] + po, xd[j] + xo, id2);
                umma_commit(&empty[s]);  // with the other issuers' commits: releases the X~ stage and P
                if (++s == stages) s = 0;
                if (++b == NB) {
                    b = 0;
                    par ^= 1u;
                }
            }
            umma_commit(d2_full);
            umma_commit(mma_done);
            mbar_drain(mma_done, 0u, status);
        }
    } else {
        // ------------------------------------------------------------------ epilogue warps
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;  // column group 0..kGroups-1
        const int row = q * 32 + lane;
        const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
        constexpr int CW = TC / kGroups;
        float2 s2 = make_float2(0.f, 0.f), s4 = make_float2(0.f, 0.f);
        float sq = 0.f;
        bool ok = true;
        for (int c = 0; c < nch; ++c) {
            const int b = c % NB;
            ok = __all_sync(0xffffffffu, mbar_wait(&d1_full[b], static_cast<uint32_t>(c / NB) & 1u, abort_flag, status));
            if (!ok) break;
            tc_fence_after();
            float v[CW];
            const uint32_t d1 = tmem + kD1Col + static_cast<uint32_t>(b * TC) + lane_off + static_cast<uint32_t>(h * CW);
            // as few loads as possible: 64-, then 32-, then 16-column pieces
            constexpr int N64 = CW / 64, N32 = (CW % 64) / 32, N16 = (CW % 32) / 16;
            static_assert(CW % 16 == 0, "column group must be a multiple of 16");
#pragma unroll
            for (int i = 0; i < N64; ++i)
                tmem_ld64(d1 + static_cast<uint32_t>(64 * i), *reinterpret_cast<float(*)[64]>(&v[64 * i]));
            if constexpr (N32 == 1) tmem_ld32(d1 + static_cast<uint32_t>(64 * N64), *reinterpret_cast<float(*)[32]>(&v[64 * N64]));
            if constexpr (N16 == 1)
                tmem_ld16(d1 + static_cast<uint32_t>(CW - 16), *reinterpret_cast<float(*)[16]>(&v[CW - 16]));
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
                if (MOMENTS || MOMENTS_ONLY) {
                    s2 = add2(s2, z2);
                    s4 = fma2(z2, z2, s4);
                }
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
                if (c >= NB) {
                    // P[b] is free once the second product of chunk c - NB retired; that product's
                    // commit released the X~ stage of chunk c - NB
                    const int cr = c - NB;
                    ok = __all_sync(0xffffffffu, mbar_wait(&empty[cr % stages], static_cast<uint32_t>(cr / stages) & 1u,
                                                           abort_flag, status));
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
        if (!MOMENTS_ONLY && ok && h < 2) {  // accumulator read-out: two warps per lane quarter
            ok = __all_sync(0xffffffffu, mbar_wait(d2_full, 0u, abort_flag, status));
            if (ok) {
                tc_fence_after();
                const int half = n_pad / 2;
                for (int g = 0; g < half / 8; ++g) {
                    const int col = h * half + g * 8;
                    float v8[8];
                    tmem_ld8(tD2 + lane_off + static_cast<uint32_t>(col), v8);
                    if constexpr (G2S == 2) {  // the odd K steps' accumulator
                        float w8[8];
                        tmem_ld8(tD2 + kD2Cols + lane_off + static_cast<uint32_t>(col), w8);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 8; ++i) v8[i] += w8[i];
                    } else {
                        tmem_ld_wait();
                    }
                    if (grow < M_act) {
                        float4* dst = reinterpret_cast<float4*>(part_acc + prow * n_pad + col);
                        dst[0] = make_float4(v8[0], v8[1], v8[2], v8[3]);
                        dst[1] = make_float4(v8[4], v8[5], v8[6], v8[7]);
                    }
                }
            }
        }
        if (h > 0) {
            float* dst = mom_sm + ((h - 1) * kTcRows + row) * 4;
            dst[0] = s2.x + s2.y;
            dst[1] = s4.x + s4.y;
            dst[2] = sq;
        }
        named_bar_sync(1, 32 * kEpiWarps);
        if (h == 0 && grow < M_act) {
            float m2 = s2.x + s2.y, m4 = s4.x + s4.y, mq = sq;
#pragma unroll
            for (int hh = 0; hh < kGroups - 1; ++hh) {  // fixed order: groups 1, 2, ...
                const float* src = mom_sm + (hh * kTcRows + row) * 4;
                m2 += src[0];
                m4 += src[1];
                mq += src[2];
            }
            part_mom[prow * 4 + 0] = m2;
            part_mom[prow * 4 + 1] = m4;
            part_mom[prow * 4 + 2] = mq;
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

template <int TC, int NB, bool MO, bool MOM>
static cudaError_t launch_tc_impl(cudaStream_t s, const CUtensorMap& xmap, const float* B32, int ldb,
                                  const int* act_idx, const int* count_dev, int M_act, int n_pad, int64_t T,
                                  int splits, int chunks_per_split, int total_chunks, float* part_acc,
                                  float* part_mom, int part_rows, int* status, int shape_ctas = 0,
                                  int* shape_out = nullptr, bool use_lo = true) {
    const TcLayout L = tc_layout(n_pad, MO, TC, NB);
    if (L.stages < static_cast<uint32_t>(NB + 1)) return cudaErrorInvalidConfiguration;
    cudaError_t e = allow_max_dyn_smem(fused_tc_kernel<TC, NB, MO, MOM>);
    if (e != cudaSuccess) return e;
    const int tiles_ub = (M_act + kTcRows - 1) / kTcRows;
    const dim3 grid = shape_ctas > 0 ? dim3(tiles_ub > shape_ctas ? tiles_ub : shape_ctas, 1)
                                     : dim3(splits, tiles_ub);
    // device-shaped launches (the fit's update loop) overlap their launch with the previous grid
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = shape_ctas > 0 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, fused_tc_kernel<TC, NB, MO, MOM>, xmap, B32, ldb, act_idx, count_dev, M_act,
                              n_pad, T, chunks_per_split, total_chunks, static_cast<int>(L.stages), L.a_bytes,
                              L.xsub_bytes, L.xstage_bytes, L.off_x, L.off_p, L.off_bar, part_acc, part_mom,
                              part_rows, status, shape_ctas, shape_out, use_lo ? 1 : 0);
}

cudaError_t launch_fused_tc_shaped(cudaStream_t s, bool moments, const CUtensorMap& xmap, const float* B32, int ldb,
                                   const int* act_idx, const int* count_dev, int M_ub, int n_pad, int64_t T, int ctas,
                                   int total_chunks, float* part_acc, float* part_mom, int* status, int* shape_out,
                                   bool use_lo) {
#define ICA_TC_SHAPED(TCV, NBV)                                                                                   \
    return moments ? launch_tc_impl<TCV, NBV, false, true>(s, xmap, B32, ldb, act_idx, count_dev, M_ub, n_pad, T, \
                                                           0, 0, total_chunks, part_acc, part_mom, 0, status,     \
                                                           ctas, shape_out, use_lo)                               \
                   : launch_tc_impl<TCV, NBV, false, false>(s, xmap, B32, ldb, act_idx, count_dev, M_ub, n_pad, T, \
                                                            0, 0, total_chunks, part_acc, part_mom, 0, status,    \
                                                            ctas, shape_out, use_lo)
    if (n_pad <= 64) ICA_TC_SHAPED(ICA_TC_SMALL_CHUNK, ICA_TC_SMALL_NB);
    if (n_pad <= 128) ICA_TC_SHAPED(128, 2);
    ICA_TC_SHAPED(64, 2);
#undef ICA_TC_SHAPED
}

cudaError_t launch_fused_tc(cudaStream_t s, bool moments_only, bool moments, const CUtensorMap& xmap, const float* B32,
                            int ldb, const int* act_idx, const int* count_dev, int M_act, int n_pad, int64_t T,
                            int splits, int chunks_per_split, int total_chunks, float* part_acc, float* part_mom,
                            int part_rows, int* status) {
#define ICA_TC_ARGS s, xmap, B32, ldb, act_idx, count_dev, M_act, n_pad, T, splits, chunks_per_split, total_chunks, \
                    part_acc, part_mom, part_rows, status
#define ICA_TC_DISPATCH(TCV, NBV)                                                                     \
    do {                                                                                            \
        if (moments_only) return launch_tc_impl<TCV, NBV, true, true>(ICA_TC_ARGS);                 \
        return moments ? launch_tc_impl<TCV, NBV, false, true>(ICA_TC_ARGS)                         \
                       : launch_tc_impl<TCV, NBV, false, false>(ICA_TC_ARGS);                       \
    } while (0)
    if (n_pad <= 64) ICA_TC_DISPATCH(ICA_TC_SMALL_CHUNK, ICA_TC_SMALL_NB);
    if (n_pad <= 128) ICA_TC_DISPATCH(128, 2);
    ICA_TC_DISPATCH(64, 2);
#undef ICA_TC_DISPATCH
#undef ICA_TC_ARGS
}

}  // namespace ica
