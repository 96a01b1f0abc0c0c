// Persistent BF16 stage of Algorithm 2: every fixed-point update of the restarts of one
// component, from the first iteration to the last, in one cooperative launch (one CTA per SM,
// all CTAs co-resident). Per iteration t:
//
//   1. update:   each CTA takes the (restart tile, sample split) that the active count gives it
//                (tc_device_shape, the same one-wave shape as the per-launch update kernel) and
//                runs the fused GEMM-cube-GEMM of Section 3.1 on the tensor cores over its
//                chunks of X~, writing its FP32 partial of (Z o Z o Z) X~^T;
//                BF16 operands (B as one or two BF16 terms, X~ BF16), or, in the FP8 form
//                (F8), E4M3 operands with power-of-two scales: the restart rows (scaled per column
//                of X~), X~ (one scale per row) and P = Z o Z o Z (one scale per restart row, from
//                the row's largest |z| of the previous iteration), FP32 accumulation and cube;
//   2. grid barrier; finish: groups of 16, 4 or 2 warps (fewer rows, larger groups) finish the
//                active rows (compensated sum of the split partials in a fixed order, b' =
//                acc / T - 3 b, normalisation, step distance, convergence flag);
//   3. grid barrier; removal of converged rows (Section 3.2): every CTA compacts the active list
//                from the flags (all CTAs compute the same list), and the loop ends when no row
//                is active or the iteration limit is reached.
//
// The arithmetic of every step is that of the per-launch path (fused_tc_kernel + finalize_kernel),
// so both give identical results, with two exceptions that change only the FP32 rounding: the
// equal work shares (opts.stage_streamk) and, at 64-sample chunks, the split first product (the
// restart rows' two BF16 terms accumulated apart and added in the epilogue). The persistent form
// removes two launches per iteration, the TMEM allocation and barrier set-up of each update, and
// the host's reads of the active count.
//
// Data written by other CTAs inside the launch (restart rows, partials, flags, the active list)
// is read with cache-global loads (L1 is not coherent across SMs). Every wait is bounded
// (ICA_WAIT_NS): on timeout the CTA raises the device status word, stops arriving at the grid
// barriers (the other CTAs then time out as well), drains its copies and MMAs, frees TMEM and
// returns.
#include "rowfin.cuh"
#include "tc_common.cuh"

namespace ica {

namespace {

struct StageArgs {
    float* B32;
    int ldb;
    int* act[2];       // the two active lists; act[cur0] holds the list on entry
    int* count[2];     // their counts
    int cur0;
    int n_pad, n;
    int64_t T;
    int total_chunks, shape_ctas;
    float* part_acc;
    float* part_mom;
    int* flags;
    int* iters;
    float* traj;  // [M][kTrajLen][2] (alpha, step distance) or null
    int* status;
    long long* rows_accum;
    unsigned int* bar_ctr;  // grid barrier counter, zero on entry
    int* ctl;               // out: iteration index reached, final active count, final list index
    int t_begin, t_end;
    float inv_T, tol;
    uint64_t wait_ns;  // limit of every wait except the teardown drains
    unsigned int stall;  // test hook: arrivals the grid barriers expect beyond the CTAs (0)
    RowProj proj;        // Algorithm 1: found components projected out of each update (none: nw = 0)
    int lo_from;         // iterations t >= lo_from add the restart rows' low BF16 term to the first product
    int streamk;         // 1: equal shares of the (tile x chunk) work when the one-wave shape leaves SMs idle
    float* zmax;         // per restart: largest |z| of its last update (for the next FP8 iteration's P scale)
    int track_until;     // iterations t with t + 1 < track_until record zmax
    const float* fp8sc;  // FP8 form: the X~ scales (see launch_fp8_copy)
    int n8;              // FP8 form: n rounded up to 32 (K of the first product, N of the second)
    int stages;
    uint32_t a_bytes, xsub_bytes, xstage_bytes, off_x, off_p, off_bar;
};

// One active row j finished by a group of R warps (warp gw of the group, named barrier bar_id):
// the split partials summed in the virtual-warp order of row_partials with V = R, the row
// completed by the group's first warp (which loads the restart row while the sums run).
// red: the group's scratch, [R][n_pad] sums, [R][n_pad] compensations, [R][4].
// Wsk > 0: the update ran in equal shares of Wsk = tiles x chunks work (see the update): row j's
// partials come from the CTAs whose shares meet its tile, in CTA order, each at row j mod 128 of
// its slot for that tile (2 k, or 2 k + 1 when its share began in the tile before).
__device__ __forceinline__ void group_finish_row(const StageArgs& a, const int* act, int j, int splits, int part_rows,
                                                 int64_t Wsk, int t, float* red, int R, int gw, int bar_id) {
    const bool want_traj = a.traj && t < kTrajLen;
    const int nq = (a.n_pad + 31) >> 5;
    int r = 0;
    float b[8];
    if (gw == 0) {
        r = __ldcg(act + j);
        load_row(a.B32, a.ldb, r, nq, a.n, b);
    }
    if (Wsk > 0) {
        const int G = static_cast<int>(gridDim.x);
        const int64_t tot = a.total_chunks;
        const int tile = j / kTcRows, rr = j % kTcRows;
        auto w0 = [&](int k) { return static_cast<int64_t>(k) * Wsk / G; };
        const int64_t first = static_cast<int64_t>(tile) * tot, last = first + tot - 1;
        int kf = static_cast<int>(first * G / Wsk), kl = static_cast<int>(last * G / Wsk);
        while (kf + 1 < G && w0(kf + 1) <= first) ++kf;
        while (kf > 0 && w0(kf) > first) --kf;
        while (kl + 1 < G && w0(kl + 1) <= last) ++kl;
        while (kl > 0 && w0(kl) > last) --kl;
        row_partials_at(a.part_acc, a.part_mom, kl - kf + 1,
                        [=](int s) {
                            const int k = kf + s;
                            const int seg = w0(k) / tot == tile ? 0 : 1;
                            return static_cast<int64_t>(2 * k + seg) * kTcRows + rr;
                        },
                        a.n_pad, want_traj, R, R, gw, red);
    } else {
        row_partials(a.part_acc, a.part_mom, splits, part_rows, a.n_pad, j, want_traj, R, R, gw, red);
    }
    named_bar_sync(bar_id, 32 * R);
    if (gw == 0) {
        float accv[8], e2, e4;
        row_combine(red, R, a.n_pad, a.n, want_traj, accv, &e2, &e4);
        finish_row_loaded(accv, b, nq, a.n, r, j, a.B32, a.ldb, a.inv_T, a.tol, a.flags, a.iters, a.traj, t,
                          want_traj, e2, e4, a.status, a.proj);
        if (a.zmax && t + 1 < a.track_until) {  // largest z^2 over the partials (slot 3) -> zmax[r]
            const int lane = threadIdx.x & 31;
            float mx = 0.f;
            if (Wsk > 0) {
                const int G = static_cast<int>(gridDim.x);
                const int64_t tot = a.total_chunks;
                const int tile = j / kTcRows, rr = j % kTcRows;
                const int64_t first = static_cast<int64_t>(tile) * tot, last = first + tot - 1;
                for (int k = lane; k < G; k += 32) {
                    const int64_t w0 = static_cast<int64_t>(k) * Wsk / G, w1 = static_cast<int64_t>(k + 1) * Wsk / G;
                    if (w1 <= first || w0 > last) continue;  // share does not meet the tile
                    const int seg = w0 / tot == tile ? 0 : 1;
                    mx = fmaxf(mx, __ldcg(a.part_mom + (static_cast<int64_t>(2 * k + seg) * kTcRows + rr) * 4 + 3));
                }
            } else {
                for (int sp = lane; sp < splits; sp += 32)
                    mx = fmaxf(mx, __ldcg(a.part_mom + (static_cast<int64_t>(sp) * part_rows + j) * 4 + 3));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) a.zmax[r] = sqrtf(mx);
        }
    }
    named_bar_sync(bar_id, 32 * R);  // the scratch is reused by the group's next row
}

}  // namespace

// F8: the FP8 form (TC = 128; xmap is then the E4M3 copy of X~, box {128, n8}).
template <int TC, int NB, bool F8>
__global__ void __launch_bounds__(kThreads, 1) stage_tc_kernel(const __grid_constant__ CUtensorMap xmap, const StageArgs a) {
    static_assert(!F8 || TC == 128, "the FP8 form uses 128-sample chunks");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    const uint32_t base_u32 = (raw_u32 + 1023u) & ~1023u;
    uint8_t* base = smem_raw + (base_u32 - raw_u32);
    constexpr uint32_t p_bytes = F8 ? 16384u : static_cast<uint32_t>(TC / 64) * 16384u;
    constexpr int G2S = F8 ? 1 : tc_g2_issuers(TC);
    // Split first product (64-sample chunks, one Z buffer): the high term's MMAs (warp 1) and the
    // low term's (warp kG2bWarp, idle as a second-product issuer at this width) go to two Z
    // accumulators from two threads, summed when the epilogue reads them. One thread issues an
    // N = 64 MMA only every 67-84 cycles, so the first product, 2 n_pad / 16 MMAs per chunk,
    // was the limit; TMEM then holds D2, Z_hi, Z_lo and B's low term (256 + 64 + 64 + 128).
    constexpr bool kSplit = !F8 && TC == 64 && NB == 1;
    static_assert(!kSplit || tc_lo_in_tmem(TC), "the split form reads B's low term from tensor memory");
    constexpr int kTeams = kSplit ? 1 : 2;  // epilogue teams taking alternate chunks
    const uint32_t stages = static_cast<uint32_t>(a.stages);
    const uint32_t sA = base_u32, sX = base_u32 + a.off_x, sP = base_u32 + a.off_p;
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + a.off_bar);
    uint64_t* full = bars;          // [8]  X~ stage loaded
    uint64_t* empty = bars + 8;     // [8]  X~ stage released by the second product that read it
    uint64_t* d1_full = bars + 16;  // [NB] Z chunk ready in TMEM
    uint64_t* d1_empty = bars + 19; // [NB] Z chunk read out by the epilogue warps
    uint64_t* p_full = bars + 22;   // [NB] P chunk written to SMEM by the epilogue warps
    uint64_t* d2_full = bars + 28;  //      accumulator complete (once per update of this CTA)
    uint64_t* mma_done = bars + 29; //      every MMA of this CTA retired (teardown)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kBars);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* mom_sm = reinterpret_cast<float*>(bars + kBars + 2);  // [3][128][4]
    int* new_count = reinterpret_cast<int*>(base + a.off_bar + 6656u);
    float* fin_scratch = reinterpret_cast<float*>(base);  // restart tile region, free while rows finish

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = static_cast<int>(gridDim.x), bid = static_cast<int>(blockIdx.x);
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], G2S);  // a commit of every second-product issuer
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(&d1_full[b], kSplit ? 2 : 1);      // a commit of every first-product issuer
            mbar_init(&d1_empty[b], kEpiWarps / kTeams);  // the epilogue team of the buffer
            mbar_init(&p_full[b], kEpiWarps / kTeams);
        }
        mbar_init(d2_full, G2S);
        mbar_init(mma_done, 1 + G2S + (kSplit ? 1 : 0));  // one commit per MMA-issuing thread
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) tma_prefetch_desc(&xmap);
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t kD2Cols = F8 ? 256u : tc_d2_cols(TC);
    constexpr uint32_t kD1Col = G2S * kD2Cols;  // Z buffers after the G2S accumulators
    constexpr uint32_t kZCols = kSplit ? 2u * TC : static_cast<uint32_t>(NB * TC);  // Z (split: Z_hi, Z_lo)
    static_assert(kD1Col + kZCols <= 512, "D2 and the Z buffers must fit in 512 TMEM columns");
    constexpr uint32_t kALoCol = kSplit ? kD1Col + kZCols : tc_alo_col(TC, NB);  // B's low term: n_pad / 2 columns
    static_assert(F8 || !tc_lo_in_tmem(TC) || kALoCol + (TC == 128 ? 64u : 128u) <= 512, "B's low term must fit TMEM");
    static_assert((kSplit ? NB == 1 : NB >= 2) && NB <= 3, "barrier slots exist for up to three Z / P buffers");

    // running counts of each role (mbarrier phases continue across the updates)
    uint32_t pc = 0;   // producer: chunks issued
    uint32_t g1c = 0;  // first-product issuer: chunks consumed
    uint32_t g1l = 0;  // low-term first-product issuer (split form): chunks consumed
    uint32_t g2c = 0;  // second-product issuer: chunks consumed
    uint32_t ec = 0;   // epilogue: chunks consumed
    uint32_t d2n = 0;  // updates this CTA took part in
    unsigned int bar_target = 0;
    int cur = a.cur0;
    int M_act = __ldcg(cur ? a.count[1] : a.count[0]);
    int t = a.t_begin;
    for (; t < a.t_end && M_act > 0; ++t) {
        const int* act = cur ? a.act[1] : a.act[0];
        int tiles, sp, cps;
        tc_device_shape(M_act, a.shape_ctas, a.total_chunks, &tiles, &sp, &cps);
        const int part_rows = tiles * kTcRows;
        const bool mom = t < kTrajLen;
        const bool use_lo = !F8 && t >= a.lo_from;
        const bool trk = a.zmax != nullptr && t + 1 < a.track_until;  // record each row's largest |z|
        // Work of this CTA: one (restart tile, sample split) of the one-wave shape, or, when that
        // shape leaves more than a sixteenth of the CTAs idle, an equal share of the (tile x
        // chunk) work in tile-major order (at most two segments: the end of one tile's chunk
        // range and the start of the next; partials per segment in slot 2 bid + segment).
        const int64_t Wsk = static_cast<int64_t>(tiles) * a.total_chunks;
        const bool sk = a.streamk && tiles * sp < (G * 15) / 16 && Wsk >= G;
        int nseg = 0, seg_tile[2] = {0, 0}, seg_c0[2] = {0, 0}, seg_nch[2] = {0, 0};
        if (!sk) {
            if (bid < tiles * sp) {
                nseg = 1;
                seg_tile[0] = bid / sp;
                seg_c0[0] = (bid % sp) * cps;
                seg_nch[0] = min(a.total_chunks, seg_c0[0] + cps) - seg_c0[0];
            }
        } else {
            const int64_t w1 = (static_cast<int64_t>(bid) + 1) * Wsk / G;
            for (int64_t w = static_cast<int64_t>(bid) * Wsk / G; w < w1 && nseg < 2;) {
                const int tl = static_cast<int>(w / a.total_chunks);
                const int64_t e = min(w1, static_cast<int64_t>(tl + 1) * a.total_chunks);
                seg_tile[nseg] = tl;
                seg_c0[nseg] = static_cast<int>(w - static_cast<int64_t>(tl) * a.total_chunks);
                seg_nch[nseg] = static_cast<int>(e - w);
                ++nseg;
                w = e;
            }
        }

        for (int seg = 0; seg < nseg; ++seg) {
        const int m0 = seg_tile[seg] * kTcRows;
        const int c_begin = seg_c0[seg];
        const int nch = seg_nch[seg];
        const int64_t prow0 = sk ? static_cast<int64_t>(2 * bid + seg) * kTcRows
                                 : static_cast<int64_t>(bid % sp) * part_rows + m0;
        if (warp >= 2 && warp < 2 + kEpiWarps) {
            if constexpr (F8) {  // restart tile -> E4M3, column k scaled by 2^(c - e_k)
                convert_restart_tile_e4m3(a.B32, a.ldb, act, m0, M_act, a.n, a.n8, sA, a.a_bytes >> 1, a.fp8sc + a.n8);
            } else {  // restart tile -> BF16 hi (shared memory) and lo (beside it, or in tensor memory)
                convert_restart_tile<tc_split_b(TC), tc_lo_in_tmem(TC)>(a.B32, a.ldb, act, m0, M_act, a.n_pad, sA,
                                                                        a.a_bytes, tmem + kALoCol, true, use_lo);
            }
            tc_fence_before();
        }
        // The restart tile is complete for the first-product issuers (warp 1, and warp kG2bWarp
        // for the low term in the split form) once the epilogue warps pass this barrier; the TMA
        // producer starts loading X~ without waiting for it.
        if ((warp >= 1 && warp < 2 + kEpiWarps) || (kSplit && warp == kG2bWarp))
            named_bar_sync(10, 32 * (1 + kEpiWarps + (kSplit ? 1 : 0)));

        {
            if (warp == 0) {
                // -------------------------------------------------------------- TMA producer
                if (lane == 0) {
                    for (int c = 0; c < nch; ++c) {
                        const uint32_t s = pc % stages;
                        if (pc >= stages &&
                            !mbar_wait(&empty[s], ((pc / stages) - 1u) & 1u, abort_flag, a.status, a.wait_ns))
                            break;
                        mbar_arrive_expect_tx(&full[s], a.xstage_bytes);
                        const int tg = (c_begin + c) * TC;
                        const uint32_t stage = sX + s * a.xstage_bytes;
                        constexpr int kBoxes = F8 ? 1 : TC / 64;  // boxes of 64 BF16 or 128 E4M3 samples
#pragma unroll
                        for (int sub = 0; sub < kBoxes; ++sub)
                            tma_load_2d(stage + static_cast<uint32_t>(sub) * a.xsub_bytes, &xmap, &full[s],
                                        tg + sub * 64, 0);
                        ++pc;
                    }
                }
            } else if (warp == 1) {
                // -------------------------------------------------------------- first products
                if (F8 && lane == 0) {
                    // E4M3: D1[128 x 128] = (A8 hi + A8 lo) (K-major, n8 entries) . X~8 chunk (MN-major, n8
                    // rows), K = 32 per MMA: K step ks at byte 32 (ks & 3) of K block ks >> 2 in A, at row
                    // 32 ks in B; the lo term's MMAs accumulate after the hi term's
                    constexpr uint32_t id1 = idesc_e4m3(128, 128, 1u);
                    const uint64_t a1_desc = sw128_desc(sA, 16u, 1024u);
                    const uint64_t b1_desc = sw128_desc(sX, a.xsub_bytes, 1024u);
                    const uint32_t stage16 = a.xstage_bytes >> 4;
                    const int ksteps1 = a.n8 / 32;
                    for (int c = 0; c < nch; ++c) {
                        const uint32_t s = g1c % stages, b = g1c % NB;
                        bool ok = mbar_wait(&full[s], (g1c / stages) & 1u, abort_flag, a.status, a.wait_ns);
                        if (ok && g1c >= static_cast<uint32_t>(NB))
                            ok = mbar_wait(&d1_empty[b], ((g1c - NB) / NB) & 1u, abort_flag, a.status, a.wait_ns);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t d1 = tmem + kD1Col + b * TC;
                        const uint64_t b1s = b1_desc + static_cast<uint64_t>(s * stage16);
#pragma unroll
                        for (int ks = 0; ks < 8; ++ks) {
                            if (ks >= ksteps1) break;
                            const uint32_t a_off = ((ks >> 2) * 16384u + (ks & 3) * 32u) >> 4;
                            const uint32_t b_off = (static_cast<uint32_t>(ks) * 4096u) >> 4;
                            umma_e4m3(d1, a1_desc + a_off, b1s + b_off, id1, ks > 0 ? 1u : 0u);
                        }
                        const uint64_t a1_lo = a1_desc + static_cast<uint64_t>((a.a_bytes >> 1) >> 4);
#pragma unroll
                        for (int ks = 0; ks < 8; ++ks) {
                            if (ks >= ksteps1) break;
                            const uint32_t a_off = ((ks >> 2) * 16384u + (ks & 3) * 32u) >> 4;
                            const uint32_t b_off = (static_cast<uint32_t>(ks) * 4096u) >> 4;
                            umma_e4m3(d1, a1_lo + a_off, b1s + b_off, id1, 1u);
                        }
                        umma_commit(&d1_full[b]);
                        ++g1c;
                    }
                } else if (!F8 && lane == 0) {
                    constexpr uint32_t id1 = idesc_bf16(128, TC, 1u);  // B: X~ MN-major
                    const uint64_t a1_desc = sw128_desc(sA, 16u, 1024u);
                    const uint64_t b1_desc = sw128_desc(sX, a.xsub_bytes, 1024u);
                    const uint32_t stage16 = a.xstage_bytes >> 4;
                    const int ksteps1 = a.n_pad / 16;
                    for (int c = 0; c < nch; ++c) {
                        const uint32_t s = g1c % stages, b = g1c % NB;
                        bool ok = mbar_wait(&full[s], (g1c / stages) & 1u, abort_flag, a.status, a.wait_ns);
                        if (ok && g1c >= static_cast<uint32_t>(NB))
                            ok = mbar_wait(&d1_empty[b], ((g1c - NB) / NB) & 1u, abort_flag, a.status, a.wait_ns);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t d1 = tmem + kD1Col + b * TC;
                        const uint64_t b1s = b1_desc + static_cast<uint64_t>(s * stage16);
#pragma unroll
                        for (int ks = 0; ks < 16; ++ks) {
                            if (ks >= ksteps1) break;
                            const uint32_t a_off = ((ks >> 2) * 16384u + (ks & 3) * 32u) >> 4;
                            const uint32_t b_off = (static_cast<uint32_t>(ks) * 2048u) >> 4;
                            umma_bf16(d1, a1_desc + a_off, b1s + b_off, id1, ks > 0 ? 1u : 0u);
                        }
                        if (!use_lo || kSplit) {  // split form: the low term's MMAs come from warp kG2bWarp
                        } else if constexpr (tc_lo_in_tmem(TC)) {
#pragma unroll
                            for (int ks = 0; ks < 16; ++ks) {
                                if (ks >= ksteps1) break;
                                const uint32_t b_off = (static_cast<uint32_t>(ks) * 2048u) >> 4;
                                umma_bf16_tmem_a_acc(d1, tmem + kALoCol + static_cast<uint32_t>(ks) * 8u, b1s + b_off, id1);
                            }
                        } else if constexpr (tc_split_b(TC)) {
                            const uint64_t a1_lo = a1_desc + static_cast<uint64_t>((a.a_bytes >> 1) >> 4);
#pragma unroll
                            for (int ks = 0; ks < 16; ++ks) {
                                if (ks >= ksteps1) break;
                                const uint32_t a_off = ((ks >> 2) * 16384u + (ks & 3) * 32u) >> 4;
                                const uint32_t b_off = (static_cast<uint32_t>(ks) * 2048u) >> 4;
                                umma_bf16_acc(d1, a1_lo + a_off, b1s + b_off, id1);
                            }
                        }
                        umma_commit(&d1_full[b]);
                        ++g1c;
                    }
                }
            } else if (kSplit && warp == kG2bWarp) {
                // -------------------------------------------------------------- first products, low term
                // Z_lo = B_lo X~ chunk (B_lo from tensor memory), for iterations that use it; other
                // iterations only arrive, so that the epilogue reads Z_hi alone
                if (lane == 0) {
                    constexpr uint32_t id1 = idesc_bf16(128, TC, 1u);
                    const uint64_t b1_desc = sw128_desc(sX, a.xsub_bytes, 1024u);
                    const uint32_t stage16 = a.xstage_bytes >> 4;
                    const int ksteps1 = a.n_pad / 16;
                    for (int c = 0; c < nch; ++c) {
                        const uint32_t s = g1l % stages;
                        bool ok = mbar_wait(&full[s], (g1l / stages) & 1u, abort_flag, a.status, a.wait_ns);
                        if (ok && g1l >= 1u) ok = mbar_wait(&d1_empty[0], (g1l - 1u) & 1u, abort_flag, a.status, a.wait_ns);
                        if (!ok) break;
                        if (use_lo) {
                            tc_fence_after();
                            const uint32_t dlo = tmem + kD1Col + TC;
                            const uint64_t b1s = b1_desc + static_cast<uint64_t>(s * stage16);
#pragma unroll
                            for (int ks = 0; ks < 16; ++ks) {
                                if (ks >= ksteps1) break;
                                const uint32_t b_off = (static_cast<uint32_t>(ks) * 2048u) >> 4;
                                umma_bf16_tmem_a(dlo, tmem + kALoCol + static_cast<uint32_t>(ks) * 8u, b1s + b_off, id1,
                                                 ks > 0 ? 1u : 0u);
                            }
                            umma_commit(&d1_full[0]);
                        } else {
                            mbar_arrive(&d1_full[0]);
                        }
                        ++g1l;
                    }
                }
            } else if (warp == kG2Warp || warp == kG2bWarp) {
                // -------------------------------------------------------------- second products
                // issuer gi of G2S: K steps j = gi mod G2S into accumulator gi
                const int gi = warp - kG2Warp;
                if (F8 && lane == 0 && gi == 0) {
                    // E4M3: D2[128 x n8] += P8 (128 x 128 samples, K-major) . X~8 chunk^T (K-major)
                    const uint32_t id2 = idesc_e4m3(128, static_cast<uint32_t>(a.n8), 0);
                    uint64_t pd[4], xd[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        pd[j] = sw128_desc(sP + static_cast<uint32_t>(j) * 32u, 16u, 1024u);
                        xd[j] = sw128_desc(sX + static_cast<uint32_t>(j) * 32u, 16u, 1024u);
                    }
                    const uint32_t stage16 = a.xstage_bytes >> 4;
                    bool ok = true;
                    for (int c = 0; c < nch; ++c) {
                        const uint32_t b = g2c % NB, s = g2c % stages;
                        ok = mbar_wait(&p_full[b], (g2c / NB) & 1u, abort_flag, a.status, a.wait_ns);
                        if (!ok) break;
                        tc_fence_after();
                        const uint64_t po = static_cast<uint64_t>((b * p_bytes) >> 4);
                        const uint64_t xo = static_cast<uint64_t>(s * stage16);
#pragma unroll
                        for (int j = 0; j < 4; ++j) umma_e4m3(tmem, pd[j] + po, xd[j] + xo, id2, (c > 0 || j > 0) ? 1u : 0u);
                        umma_commit(&empty[s]);  // releases the stage and P
                        ++g2c;
                    }
                    if (ok) umma_commit(d2_full);
                } else if (!F8 && lane == 0 && gi < G2S) {
                    const uint32_t id2 = idesc_bf16(128, static_cast<uint32_t>(a.n_pad), 0);
                    const uint32_t dacc = tmem + static_cast<uint32_t>(gi) * kD2Cols;
                    constexpr int KSI = TC / 16 / G2S;  // K steps of this issuer: gi, gi + G2S, ...
                    uint64_t pd[KSI], xd[KSI];
#pragma unroll
                    for (int j = 0; j < KSI; ++j) {
                        const uint32_t ks = static_cast<uint32_t>(gi + j * G2S);
                        pd[j] = sw128_desc(sP + (ks >> 2) * 16384u + (ks & 3u) * 32u, 16u, 1024u);
                        xd[j] = sw128_desc(sX + (ks >> 2) * a.xsub_bytes + (ks & 3u) * 32u, 16u, 1024u);
                    }
                    const uint32_t stage16 = a.xstage_bytes >> 4;
                    bool ok = true;
                    for (int c = 0; c < nch; ++c) {
                        const uint32_t b = g2c % NB, s = g2c % stages;
                        ok = mbar_wait(&p_full[b], (g2c / NB) & 1u, abort_flag, a.status, a.wait_ns);
                        if (!ok) break;
                        tc_fence_after();
                        const uint64_t po = static_cast<uint64_t>((b * p_bytes) >> 4);
                        const uint64_t xo = static_cast<uint64_t>(s * stage16);
                        umma_bf16(dacc, pd[0] + po, xd[0] + xo, id2, c > 0 ? 1u : 0u);
#pragma unroll
                        for (int j = 1; j < KSI; ++j) umma_bf16_acc(dacc, pd[j] + po, xd[j] + xo, id2);
                        umma_commit(&empty[s]);  // with the other issuers' commits: releases the stage and P
                        ++g2c;
                    }
                    if (ok) umma_commit(d2_full);
                }
            } else {
                // -------------------------------------------------------------- epilogue warps
                // Two teams of 8 warps take alternate chunks (team k: chunks g = k mod 2, Z / P
                // buffer k), so that one team's TMEM-load and barrier latency overlaps the other
                // team's cube conversion. In a team, warp (lane quarter q, half hh) converts rows
                // 32q.. of columns [hh TC/2, (hh+1) TC/2) in two passes of TC/4 columns. The split
                // form has one Z / P buffer and one team of 16 warps: warp (q, h) converts columns
                // [h TC/4, (h+1) TC/4) of every chunk, Z_hi + Z_lo, in one pass.
                static_assert(kSplit || NB == 2, "one Z / P buffer per epilogue team");
                constexpr int kPasses = kSplit ? 1 : 2;
                const int q = warp & 3;
                const int h = (warp - 2) >> 2;  // moment group 0..3 = 2 team + hh
                const int team = h >> 1, hh = h & 1;
                const int row = q * 32 + lane;
                const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
                constexpr int CW = TC / 4;  // columns per pass
                float2 s2 = make_float2(0.f, 0.f), s4 = make_float2(0.f, 0.f);
                float z2max = 0.f;  // largest z^2 of this thread's entries (trk)
                // FP8 form: z = D1 2^-c; P = e4m3(v z^3) with the row's scale v = 2^e, the largest
                // power of two with v (2 zmax)^3 <= 448 (zmax: the row's largest |z| of the previous
                // iteration; the factor 2 leaves room for the row's change since then)
                int ev = 0;  // v = 2^ev
                if constexpr (F8) {
                    if (m0 + row < M_act) {
                        const float zm = __ldcg(a.zmax + __ldcg(act + m0 + row));
                        ev = pow2_fit_exponent(8.f * zm * zm * zm, 448.f);
                    }
                }
                bool ok = true;
                for (int c = 0; c < nch && ok; ++c) {
                    const uint32_t g = ec + static_cast<uint32_t>(c);
                    if (kTeams == 2 && static_cast<int>(g & 1u) != team) continue;
                    const uint32_t b = g % NB;
                    ok = __all_sync(0xffffffffu, mbar_wait(&d1_full[b], (g / NB) & 1u, abort_flag, a.status, a.wait_ns));
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t pbase = sP + b * p_bytes;
#pragma unroll 1
                    for (int pass = 0; pass < kPasses; ++pass) {
                        const int col0 = kSplit ? h * CW : hh * (TC / 2) + pass * CW;  // first sample of this pass
                        float v[CW];
                        const uint32_t d1 = tmem + kD1Col + b * TC + lane_off + static_cast<uint32_t>(col0);
                        constexpr int N64 = CW / 64, N32 = (CW % 64) / 32, N16 = (CW % 32) / 16;
                        static_assert(CW % 16 == 0, "column group must be a multiple of 16");
#pragma unroll
                        for (int i = 0; i < N64; ++i)
                            tmem_ld64(d1 + static_cast<uint32_t>(64 * i), *reinterpret_cast<float(*)[64]>(&v[64 * i]));
                        if constexpr (N32 == 1)
                            tmem_ld32(d1 + static_cast<uint32_t>(64 * N64),
                                      *reinterpret_cast<float(*)[32]>(&v[64 * N64]));
                        if constexpr (N16 == 1)
                            tmem_ld16(d1 + static_cast<uint32_t>(CW - 16), *reinterpret_cast<float(*)[16]>(&v[CW - 16]));
                        if constexpr (kSplit) {  // + the low term's accumulator
                            static_assert(CW == 16, "split form: 16 columns per warp");
                            if (use_lo) {
                                float w[16];
                                tmem_ld16(d1 + static_cast<uint32_t>(TC), w);
                                tmem_ld_wait();
#pragma unroll
                                for (int i = 0; i < 16; ++i) v[i] += w[i];
                            }
                        }
                        tmem_ld_wait();
                        if (pass == kPasses - 1) {  // the team has read all of Z(g)
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&d1_empty[b]);
                        }
                        uint32_t pk[CW / 2];
                        if constexpr (F8) {
                            const float dz = __ldg(a.fp8sc + 3 * a.n8), vr = ldexpf(1.f, ev);
#pragma unroll
                            for (int i = 0; i < CW; i += 4) {
                                float2 p[2];
#pragma unroll
                                for (int h2 = 0; h2 < 2; ++h2) {
                                    const float2 z = mul2(make_float2(v[i + 2 * h2], v[i + 2 * h2 + 1]), make_float2(dz, dz));
                                    const float2 z2 = mul2(z, z);
                                    s2 = add2(s2, z2);
                                    s4 = fma2(z2, z2, s4);
                                    z2max = fmaxf(z2max, fmaxf(z2.x, z2.y));
                                    p[h2] = mul2(mul2(z2, z), make_float2(vr, vr));
                                }
                                pk[i / 4] = pack_e4m3x4(p[0].x, p[0].y, p[1].x, p[1].y);
                            }
                        } else if (mom && trk) {
#pragma unroll
                            for (int i = 0; i < CW; i += 2) {
                                const float2 z = make_float2(v[i], v[i + 1]);
                                const float2 z2 = mul2(z, z);
                                s2 = add2(s2, z2);
                                s4 = fma2(z2, z2, s4);
                                z2max = fmaxf(z2max, fmaxf(z2.x, z2.y));
                                const float2 z3 = mul2(z2, z);
                                pk[i / 2] = pack_bf16x2(z3.x, z3.y);
                            }
                        } else if (mom) {
#pragma unroll
                            for (int i = 0; i < CW; i += 2) {
                                const float2 z = make_float2(v[i], v[i + 1]);
                                const float2 z2 = mul2(z, z);
                                s2 = add2(s2, z2);
                                s4 = fma2(z2, z2, s4);
                                const float2 z3 = mul2(z2, z);
                                pk[i / 2] = pack_bf16x2(z3.x, z3.y);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < CW; i += 2) {
                                const float2 z = make_float2(v[i], v[i + 1]);
                                const float2 z3 = mul2(mul2(z, z), z);
                                pk[i / 2] = pack_bf16x2(z3.x, z3.y);
                            }
                        }
                        if (pass == 0 && g >= static_cast<uint32_t>(NB)) {
                            // P[b] is free once the second product of chunk g - NB retired
                            const uint32_t cr = g - NB;
                            ok = __all_sync(0xffffffffu,
                                            mbar_wait(&empty[cr % stages], (cr / stages) & 1u, abort_flag, a.status, a.wait_ns));
                            if (!ok) break;
                        }
                        constexpr int kPer16 = F8 ? 16 : 8;  // samples per 16-byte chunk of P
#pragma unroll
                        for (int j = 0; j < CW / kPer16; ++j) {
                            const int col = col0 + j * kPer16;  // sample within the chunk
                            const uint32_t addr =
                                F8 ? pbase + sw128_off(static_cast<uint32_t>(row), static_cast<uint32_t>(col >> 4))
                                   : pbase + static_cast<uint32_t>(col >> 6) * 16384u +
                                         sw128_off(static_cast<uint32_t>(row), static_cast<uint32_t>((col & 63) >> 3));
                            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(pk[j * 4 + 0]),
                                         "r"(pk[j * 4 + 1]), "r"(pk[j * 4 + 2]), "r"(pk[j * 4 + 3])
                                         : "memory");
                        }
                    }
                    if (!ok) break;
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&p_full[b]);
                }
                ec += static_cast<uint32_t>(nch);
                const int grow = m0 + row;
                const int64_t prow = prow0 + row;
                if (ok && h < 2) {  // accumulator read-out: two warps per lane quarter
                    ok = __all_sync(0xffffffffu, mbar_wait(d2_full, d2n & 1u, abort_flag, a.status, a.wait_ns));
                    if (ok) {
                        tc_fence_after();
                        const int half = a.n_pad / 2;
                        for (int g = 0; g < half / 8; ++g) {
                            const int col = h * half + g * 8;
                            float v8[8];
                            tmem_ld8(tmem + lane_off + static_cast<uint32_t>(col), v8);
                            if constexpr (G2S == 2) {  // the odd K steps' accumulator
                                float w8[8];
                                tmem_ld8(tmem + kD2Cols + lane_off + static_cast<uint32_t>(col), w8);
                                tmem_ld_wait();
#pragma unroll
                                for (int i = 0; i < 8; ++i) v8[i] += w8[i];
                            } else {
                                tmem_ld_wait();
                            }
                            if constexpr (F8) {  // undo the scales of P (row) and X~ (column): exact
                                const float4* isx = reinterpret_cast<const float4*>(a.fp8sc + 2 * a.n8 + col);
                                const float4 i0 = __ldg(isx), i1 = __ldg(isx + 1);
                                const float is[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
                                const float inv_vr = ldexpf(1.f, -ev);
#pragma unroll
                                for (int i = 0; i < 8; ++i) v8[i] *= inv_vr * is[i];
                            }
                            if (grow < M_act) {
                                float4* dst = reinterpret_cast<float4*>(a.part_acc + prow * a.n_pad + col);
                                dst[0] = make_float4(v8[0], v8[1], v8[2], v8[3]);
                                dst[1] = make_float4(v8[4], v8[5], v8[6], v8[7]);
                            }
                        }
                    }
                }
                ++d2n;
                if (h > 0) {
                    float* dst = mom_sm + ((h - 1) * kTcRows + row) * 4;
                    dst[0] = s2.x + s2.y;
                    dst[1] = s4.x + s4.y;
                    dst[2] = 0.f;
                    dst[3] = z2max;
                }
                named_bar_sync(1, 32 * kEpiWarps);
                if (h == 0 && grow < M_act) {
                    float m2 = s2.x + s2.y, m4 = s4.x + s4.y, mq = 0.f, mx = z2max;
#pragma unroll
                    for (int hh = 0; hh < kGroups - 1; ++hh) {  // fixed order: groups 1, 2, ...
                        const float* src = mom_sm + (hh * kTcRows + row) * 4;
                        m2 += src[0];
                        m4 += src[1];
                        mq += src[2];
                        mx = fmaxf(mx, src[3]);
                    }
                    a.part_mom[prow * 4 + 0] = m2;
                    a.part_mom[prow * 4 + 1] = m4;
                    a.part_mom[prow * 4 + 2] = mq;
                    a.part_mom[prow * 4 + 3] = mx;  // largest z^2 of the partial's samples
                }
            }
        }
        }  // segments
        // ---------------------------------------------------------------- finish the rows
        tc_fence_before();
        bar_target += static_cast<unsigned int>(G);
        if (!grid_barrier(a.bar_ctr, bar_target + a.stall, abort_flag, a.status, a.wait_ns)) break;
        tc_fence_after();
        if (warp < 16) {  // groups of R warps, one row per group and round (fin_vwarps)
            const int R = fin_vwarps(M_act, G), ngrp = 16 / R;
            const int grp = warp / R, gw = warp % R;
            float* red = fin_scratch + grp * R * (2 * a.n_pad + 4);
            for (int j = bid * ngrp + grp; j < M_act; j += G * ngrp)
                group_finish_row(a, act, j, sp, part_rows, sk ? Wsk : 0, t, red, R, gw, 2 + grp);
        }
        bar_target += static_cast<unsigned int>(G);
        if (!grid_barrier(a.bar_ctr, bar_target + a.stall, abort_flag, a.status, a.wait_ns)) break;
        // ---------------------------------------------------------------- remove converged rows
        compact_block(a.flags, act, M_act, cur ? a.act[0] : a.act[1], new_count, bid == 0 ? a.rows_accum : nullptr, kThreads);
        __syncthreads();
        const int M_new = *reinterpret_cast<volatile int*>(new_count);
        __syncthreads();  // new_count is rewritten by the next compaction
        cur ^= 1;
        M_act = M_new;
    }
    // ------------------------------------------------------------------ teardown
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && lane == 0) {  // every issued load must land before the CTA exits
        for (uint32_t s = 0; s < stages && s < pc; ++s) {
            const uint32_t c_last = s + ((pc - 1u - s) / stages) * stages;
            mbar_drain(&full[s], (c_last / stages) & 1u, a.status);
        }
    }
    if ((warp == 1 || warp == kG2Warp || (warp == kG2bWarp && (G2S == 2 || kSplit))) && lane == 0) {
        umma_commit(mma_done);
        mbar_drain(mma_done, 0u, a.status);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
    if (bid == 0 && threadIdx.x == 0 && !*abort_flag) {
        a.ctl[0] = t;
        a.ctl[1] = M_act;
        a.ctl[2] = cur;
        *(cur ? a.count[1] : a.count[0]) = M_act;
    }
}

template <int TC, int NB, bool F8>
static cudaError_t launch_stage_impl(cudaStream_t s, const CUtensorMap& xmap, const StageLaunch& p,
                                     int* resident) {
    const int n8 = (p.n + 31) / 32 * 32;
    const TcLayout L = F8 ? tc_layout_e4m3(n8, p.n_pad, 1024u)  // + the compaction's static scratch
                          : tc_layout(p.n_pad, false, TC, NB, 1024u);
    if (L.stages < static_cast<uint32_t>(NB + 1)) return cudaErrorInvalidConfiguration;
    if (F8 && (!p.fp8sc || !p.zmax || n8 > 256)) return cudaErrorInvalidValue;
    cudaError_t e = allow_max_dyn_smem(stage_tc_kernel<TC, NB, F8>);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_tc_kernel<TC, NB, F8>, kThreads, L.total)) !=
        cudaSuccess)
        return e;
    if (resident) *resident = per_sm * sms;
    if (per_sm * sms < p.ctas) return cudaErrorCooperativeLaunchTooLarge;  // nothing launched
    StageArgs a{};
    a.B32 = p.B32;
    a.ldb = p.ldb;
    a.act[0] = p.act0;
    a.act[1] = p.act1;
    a.count[0] = p.count0;
    a.count[1] = p.count1;
    a.cur0 = p.cur0;
    a.n_pad = p.n_pad;
    a.n = p.n;
    a.T = p.T;
    a.total_chunks = static_cast<int>((p.T + TC - 1) / TC);
    a.shape_ctas = p.ctas;
    a.part_acc = p.part_acc;
    a.part_mom = p.part_mom;
    a.flags = p.flags;
    a.iters = p.iters;
    a.traj = p.traj;
    a.status = p.status;
    a.rows_accum = p.rows_accum;
    a.bar_ctr = p.bar_ctr;
    a.ctl = p.ctl;
    a.t_begin = p.t_begin;
    a.t_end = p.t_end;
    a.inv_T = static_cast<float>(p.inv_T);
    a.tol = static_cast<float>(p.tol);
    a.wait_ns = p.wait_ns ? p.wait_ns : ICA_WAIT_NS;
    a.stall = p.stall ? 1u : 0u;
    a.proj = RowProj{p.Wp, p.Wp ? p.nw : 0, p.ldw};
    a.lo_from = p.lo_from;
    a.streamk = p.streamk;
    a.zmax = p.zmax;
    a.track_until = p.zmax ? p.track_until : 0;
    a.fp8sc = p.fp8sc;
    a.n8 = n8;
    a.stages = static_cast<int>(L.stages);
    a.a_bytes = L.a_bytes;
    a.xsub_bytes = L.xsub_bytes;
    a.xstage_bytes = L.xstage_bytes;
    a.off_x = L.off_x;
    a.off_p = L.off_p;
    a.off_bar = L.off_bar;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(p.ctas), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, stage_tc_kernel<TC, NB, F8>, xmap, a);
}

cudaError_t launch_stage_tc(cudaStream_t s, const CUtensorMap& xmap, const StageLaunch& p, int* resident) {
    if (p.fp8) return launch_stage_impl<128, 2, true>(s, xmap, p, resident);
    if (p.n_pad <= 64) return launch_stage_impl<ICA_TC_SMALL_CHUNK, ICA_TC_SMALL_NB, false>(s, xmap, p, resident);
    if (p.n_pad <= 128) return launch_stage_impl<128, 2, false>(s, xmap, p, resident);
    return launch_stage_impl<64, 1, false>(s, xmap, p, resident);  // the split first product
}

}  // namespace ica
