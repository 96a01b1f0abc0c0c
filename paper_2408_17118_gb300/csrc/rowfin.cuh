// Row completion, active-list compaction and the grid barrier shared by the finalize kernel and
// the persistent stage and refinement kernels (one update of Section 3.1 / removal of Section 3.2).
#pragma once

#include "common.cuh"
#include "internal.h"

namespace ica {

struct CompSum {  // s + c carries the exact running sum to about twice FP32 precision
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ float value() const { return s + c; }
};

// Restart row r's current entries (lane's columns k = lane + 32 q), loaded ahead of the split
// sums so that their latency overlaps them. Cache-global loads: in the persistent stage kernel
// other CTAs wrote these rows earlier in the same launch.
__device__ __forceinline__ void load_row(const float* __restrict__ B32, int ldb, int r, int nq, int n, float (&b)[8]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k = lane + 32 * q;
        b[q] = (q < nq && k < n) ? __ldcg(B32 + static_cast<int64_t>(r) * ldb + k) : 0.f;
    }
}

// Projection of Algorithm 1 (FastICA with deflation on the full whitened data): the found
// components W (nw rows of ld floats, FP32 copy) are projected out of each update,
// w <- w - W^T (W w). nw = 0 for Algorithm 2, whose reduced rows need no projection.
struct RowProj {
    const float* W;
    int nw, ld;
};

// One warp finishes active row j (restart r, current entries b) from the summed update u*T
// (acc): b' = acc / T - 3 b (Algorithm 1: then projected, RowProj), normalisation, distance,
// flag, iteration count and trajectory.
__device__ __forceinline__ void finish_row_loaded(const float (&accv)[8], const float (&b)[8], int nq, int n, int r,
                                                  int j, float* __restrict__ B32, int ldb, float inv_T, float tol,
                                                  int* __restrict__ flags, int* __restrict__ iters,
                                                  float* __restrict__ traj, int t_iter, bool want_traj, float e2sum,
                                                  float e4sum, int* status, RowProj proj = RowProj{nullptr, 0, 0}) {
    const int lane = threadIdx.x & 31;
    float u[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k = lane + 32 * q;
        u[q] = (q < nq && k < n) ? accv[q] * inv_T - 3.f * b[q] : 0.f;
    }
    for (int i = 0; i < proj.nw; ++i) {  // u -= w_i (w_i . u), w_i in turn (modified Gram-Schmidt)
        const float* wi = proj.W + static_cast<int64_t>(i) * proj.ld;
        float d = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = lane + 32 * q;
            if (q < nq && k < n) d = fmaf(__ldcg(wi + k), u[q], d);
        }
        d = warp_sumf(d);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = lane + 32 * q;
            if (q < nq && k < n) u[q] = fmaf(-d, __ldcg(wi + k), u[q]);
        }
    }
    float ss = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) ss = fmaf(u[q], u[q], ss);
    ss = warp_sumf(ss);
    const bool bad = !(ss > 0.f) || !isfinite(ss);
    float dm = 0.f, dp = 0.f;
    const float inv = bad ? 0.f : rsqrtf(ss);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        u[q] *= inv;
        dm = fmaf(u[q] - b[q], u[q] - b[q], dm);
        dp = fmaf(u[q] + b[q], u[q] + b[q], dp);
    }
    dm = warp_sumf(dm);
    dp = warp_sumf(dp);
    const float d = sqrtf(fminf(dm, dp));
    if (!bad) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = lane + 32 * q;
            if (q < nq && k < n) B32[static_cast<int64_t>(r) * ldb + k] = u[q];
        }
    }
    if (lane == 0) {
        flags[j] = (!bad && d > tol) ? 1 : 0;
        iters[r] = __ldcg(iters + r) + 1;
        if (bad) atomicOr(status, DEV_NONFINITE);
        if (want_traj) {
            const float e2 = e2sum * inv_T, e4 = e4sum * inv_T;
            const float alpha = e2 > 0.f ? e4 / (e2 * e2) - 3.f : 0.f;
            traj[(static_cast<int64_t>(r) * kTrajLen + t_iter) * 2 + 0] = alpha;
            traj[(static_cast<int64_t>(r) * kTrajLen + t_iter) * 2 + 1] = d;
        }
    }
}

// Compensated sums of active row j's split partials in the virtual-warp order: virtual warp v
// of V adds splits v, v + V, v + 2V, ... in increasing order (and, with moments, their sum z^2
// and sum z^4); the V partial sums are then combined in the order v = 0, 1, ..., V - 1
// (row_combine). A group of R real warps (warp w of the group) computes virtual warps w,
// w + R, ... into red: [V][n_pad] sums, [V][n_pad] compensations, [V][4] moment sums.
// General form: partial s of the row sits at row index prow_of(s) of part_acc / part_mom.
template <typename RowOf>
__device__ __forceinline__ void row_partials_at(const float* __restrict__ part_acc, const float* __restrict__ part_mom,
                                                int splits, RowOf prow_of, int n_pad, bool want_mom, int V, int R,
                                                int w, float* red) {
    const int lane = threadIdx.x & 31;
    const int nq = (n_pad + 31) >> 5;
    float* red_s = red;
    float* red_c = red + V * n_pad;
    float* redm = red + 2 * V * n_pad;
    for (int v = w; v < V; v += R) {
        CompSum acc[8];
        CompSum m2, m4;
#pragma unroll 8
        for (int sp = v; sp < splits; sp += V) {
            const int64_t prow = prow_of(sp);
            const float* p = part_acc + prow * n_pad;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q >= nq) break;
                const int k = lane + 32 * q;
                if (k < n_pad) acc[q].add(__ldcg(p + k));
            }
            if (want_mom && lane == 0) {
                m2.add(__ldcg(part_mom + prow * 4 + 0));
                m4.add(__ldcg(part_mom + prow * 4 + 1));
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q >= nq) break;
            const int k = lane + 32 * q;
            if (k < n_pad) {
                red_s[v * n_pad + k] = acc[q].s;
                red_c[v * n_pad + k] = acc[q].c;
            }
        }
        if (lane == 0) {
            redm[4 * v + 0] = m2.s;
            redm[4 * v + 1] = m2.c;
            redm[4 * v + 2] = m4.s;
            redm[4 * v + 3] = m4.c;
        }
    }
}

// Split layout: partial s of active row j at row s * part_rows + j.
__device__ __forceinline__ void row_partials(const float* __restrict__ part_acc, const float* __restrict__ part_mom,
                                             int splits, int part_rows, int n_pad, int j, bool want_mom, int V,
                                             int R, int w, float* red) {
    row_partials_at(part_acc, part_mom, splits,
                    [=](int sp) { return static_cast<int64_t>(sp) * part_rows + j; }, n_pad, want_mom, V, R, w,
                    red);
}

// One warp combines the V virtual-warp sums of row_partials (after a barrier of the group).
__device__ __forceinline__ void row_combine(const float* red, int V, int n_pad, int n, bool want_mom, float (&accv)[8],
                                            float* e2sum, float* e4sum) {
    const int lane = threadIdx.x & 31;
    const int nq = (n_pad + 31) >> 5;
    const float* red_s = red;
    const float* red_c = red + V * n_pad;
    const float* redm = red + 2 * V * n_pad;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k = lane + 32 * q;
        accv[q] = 0.f;
        if (q < nq && k < n) {
            CompSum acc;
            float cs = 0.f;
            for (int ww = 0; ww < V; ++ww) {
                acc.add(red_s[ww * n_pad + k]);
                cs += red_c[ww * n_pad + k];
            }
            accv[q] = acc.value() + cs;
        }
    }
    CompSum m2, m4;
    if (want_mom)
        for (int ww = 0; ww < V; ++ww) {
            m2.add(redm[4 * ww + 0]);
            m2.add(redm[4 * ww + 1]);
            m4.add(redm[4 * ww + 2]);
            m4.add(redm[4 * ww + 3]);
        }
    *e2sum = m2.value();
    *e4sum = m4.value();
}

// Grid-wide barrier over the CTAs of a cooperative launch: arrival counter with release (fence +
// red.release) and a bounded acquire spin by one thread. `target` is the number of arrivals of all
// barriers so far. Returns false (and raises the abort flag) when the arrivals do not reach the
// target within limit_ns.
__device__ __forceinline__ bool grid_barrier(unsigned int* ctr, unsigned int target, volatile int* abort_flag,
                                             int* status, uint64_t limit_ns = ICA_WAIT_NS) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!*abort_flag) {
            __threadfence();
            asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(ctr), "r"(1u) : "memory");
            const uint64_t t0 = global_ns();
            for (uint32_t it = 0;; ++it) {
                unsigned int seen;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(ctr) : "memory");
                if (seen >= target) break;
                if ((it & 15u) == 15u && global_ns() - t0 > limit_ns) {
                    atomicOr(status, DEV_TIMEOUT);
                    *abort_flag = 1;
                    break;
                }
            }
            __threadfence();
        }
    }
    __syncthreads();
    return !*abort_flag;
}

// Stable compaction of the active list (Section 3.2: converged rows leave B) by one block of
// nthr threads (at most 32 warps): act_out/count_out receive the rows whose flag is set, in
// order; rows_accum (optional) accumulates the rows the iteration updated. The flags were written
// by other blocks: read through L2. Called by every thread of the block.
__device__ __forceinline__ void compact_block(const int* __restrict__ flags, const int* __restrict__ act_idx,
                                              int M_act, int* __restrict__ act_out, int* count_out,
                                              long long* rows_accum, int nthr) {
    __shared__ int warp_tot[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per = (M_act + nthr - 1) / nthr;
    const int b0 = threadIdx.x * per, e0 = min(M_act, b0 + per);
    int local = 0;
    for (int i = b0; i < e0; ++i) local += __ldcg(flags + i) != 0;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    int before = 0;
    for (int ww = 0; ww < w; ++ww) before += warp_tot[ww];
    int pos = before + incl - local;
    for (int i = b0; i < e0; ++i)
        if (__ldcg(flags + i)) act_out[pos++] = act_idx ? __ldcg(act_idx + i) : i;
    if (threadIdx.x == nthr - 1) {
        *count_out = before + incl;
        if (rows_accum) *rows_accum += M_act;  // rows this iteration updated
    }
}

// The last of the `blocks` participating blocks to finish (each counts itself in after its flags
// are visible device-wide) compacts the active list into act_out/count_out; *done_ctr is zero on
// entry and is left zero. act_out and count_out must not alias the input list and count.
template <int NW>
__device__ __forceinline__ void compact_tail(const int* __restrict__ flags, const int* __restrict__ act_idx,
                                             int M_act, int* __restrict__ act_out, int* count_out,
                                             long long* rows_accum, unsigned int* done_ctr, int blocks) {
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        is_last = atomicAdd(done_ctr, 1u) == static_cast<unsigned>(blocks - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    compact_block(flags, act_idx, M_act, act_out, count_out, rows_accum, NW * 32);
    if (threadIdx.x == 0) *done_ctr = 0u;  // ready for the next launch
}

}  // namespace ica
