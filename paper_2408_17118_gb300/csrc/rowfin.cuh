// Row completion and active-list compaction shared by the finalize kernel and the fused
// tcgen05 kernel's split reduction (one update of Section 3.1 / removal of Section 3.2).
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

// Warp 0 of a block (or the row's own warp) finishes row j from the summed update u*T (acc):
// b' = acc / T - 3 b, normalisation, distance, flag, iteration count and trajectory.
__device__ __forceinline__ void finish_row(const float (&accv)[8], int nq, int n, const int* __restrict__ act_idx,
                                           int j, float* __restrict__ B32, int ldb, float inv_T, float tol,
                                           int* __restrict__ flags, int* __restrict__ iters,
                                           float* __restrict__ traj, int t_iter, bool want_traj, float e2sum,
                                           float e4sum, int* status) {
    const int lane = threadIdx.x & 31;
    const int r = act_idx ? act_idx[j] : j;
    float u[8], b[8];
    float ss = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k = lane + 32 * q;
        u[q] = 0.f;
        b[q] = 0.f;
        if (q < nq && k < n) {
            b[q] = B32[static_cast<int64_t>(r) * ldb + k];
            u[q] = accv[q] * inv_T - 3.f * b[q];
            ss = fmaf(u[q], u[q], ss);
        }
    }
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
        iters[r] += 1;
        if (bad) atomicOr(status, DEV_NONFINITE);
        if (want_traj) {
            const float e2 = e2sum * inv_T, e4 = e4sum * inv_T;
            const float alpha = e2 > 0.f ? e4 / (e2 * e2) - 3.f : 0.f;
            traj[(static_cast<int64_t>(r) * kTrajLen + t_iter) * 2 + 0] = alpha;
            traj[(static_cast<int64_t>(r) * kTrajLen + t_iter) * 2 + 1] = d;
        }
    }
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
        if (__ldcg(flags + i)) act_out[pos++] = act_idx ? act_idx[i] : i;
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
