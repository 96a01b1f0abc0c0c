// Per-restart kernels of the fast ordering ICA (Algorithm 2): initial restarts, the
// normalise / converge / remove step (Section 3.2), stream compaction of the active rows,
// kurtosis and Upsilon of candidates (Eq. 1-2), candidate selection, and the append
// w_i = b_p G of the winner.
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "rowfin.cuh"

namespace ica {

// ------------------------------------------------------------------------------------------
// Initial restarts (Algorithm 2: "Initialize B as an L x (N-i+1) random matrix", then every
// row normalised). One warp per restart row; lane j handles column pairs (2j, 2j+1) for
// j = lane + 32q. Values come from Philox4x32-10 + Box-Muller in FP64, or from a caller B0.
// ------------------------------------------------------------------------------------------
__global__ void init_restarts_kernel(uint64_t seed, int comp, int M, int n, int ldb, const float* __restrict__ B0,
                                     int B0_ld, float* __restrict__ B) {
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (l >= M) return;
    double v[8];
    double ss = 0.0;
    const uint2 key = make_uint2(static_cast<uint32_t>(seed & 0xffffffffu), static_cast<uint32_t>(seed >> 32));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = lane + 32 * q;
        double z0 = 0.0, z1 = 0.0;
        if (2 * j < n) {
            if (B0) {
                z0 = B0[static_cast<int64_t>(l) * B0_ld + 2 * j];
                if (2 * j + 1 < n) z1 = B0[static_cast<int64_t>(l) * B0_ld + 2 * j + 1];
            } else {
                const uint4 r = philox4x32_10(make_uint4(static_cast<uint32_t>(j), static_cast<uint32_t>(l),
                                                         static_cast<uint32_t>(comp), 0u),
                                              key);
                const double u1 = uniform52(r.x, r.y);
                const double u2 = uniform52(r.z, r.w);
                const double rad = sqrt(-2.0 * log(u1));
                const double th = 6.283185307179586 * u2;
                z0 = rad * cos(th);
                if (2 * j + 1 < n) z1 = rad * sin(th);
            }
        }
        v[2 * q] = z0;
        v[2 * q + 1] = z1;
        ss += z0 * z0 + z1 * z1;
    }
    ss = warp_sum(ss);
    const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = 2 * (lane + 32 * q);
        if (c < ldb) B[static_cast<int64_t>(l) * ldb + c] = static_cast<float>(v[2 * q] * inv);
        if (c + 1 < ldb) B[static_cast<int64_t>(l) * ldb + c + 1] = static_cast<float>(v[2 * q + 1] * inv);
    }
}

cudaError_t launch_init_restarts(cudaStream_t s, uint64_t seed, int comp, int M, int n, int ldb, const float* B0,
                                 int B0_ld, float* B) {
    const int threads = 256;
    const int blocks = (M * 32 + threads - 1) / threads;
    init_restarts_kernel<<<blocks, threads, 0, s>>>(seed, comp, M, n, ldb, B0, B0_ld, B);
    return cudaGetLastError();
}

__global__ void iota_kernel(int* idx, int count, int* count_dev) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) idx[i] = i;
    if (i == 0 && count_dev) *count_dev = count;
}
cudaError_t launch_iota(cudaStream_t s, int* idx, int count, int* count_dev) {
    iota_kernel<<<(count + 255) / 256, 256, 0, s>>>(idx, count, count_dev);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Normalise / converge / remove (Algorithm 2 inner loop; Section 3.2). One CTA of NW warps per
// active row j (restart r = act_idx[j]); rows j >= *count_dev exit (the grid is sized for an
// upper bound). The split-T partial sums of (Z o Z o Z) X~^T are added deterministically: warp w
// sums splits w, w + NW, ... in order, then warp 0 adds the NW warp sums in order. Then
// b' = acc / T - 3 b, b' <- b' / ||b'||, d = min(||b' - b||, ||b' + b||); the row stays active
// iff d > tol. Rows whose update is zero or non-finite are retired and flagged in the status
// word. For the first kTrajLen iterations the kurtosis of the pre-update row and d are kept as
// per-restart features.
// All arithmetic is FP32 (GB300's FP64 rate is 1/64 of FP32 and this kernel runs every
// iteration); the sums over splits are compensated (Neumaier), so their error stays at one FP32
// rounding of the result instead of growing with the number of splits.
// ------------------------------------------------------------------------------------------
// One row j of the update: all NW warps sum the split partials, warp 0 finishes the row.
template <int NW>
__device__ __forceinline__ void finalize_row(const float* __restrict__ part_acc, const float* __restrict__ part_mom,
                                             int splits, int part_rows, int n_pad, int n,
                                             const int* __restrict__ act_idx, int j, float* __restrict__ B32,
                                             int ldb, float inv_T, float tol, int* __restrict__ flags,
                                             int* __restrict__ iters, float* __restrict__ traj, int t_iter,
                                             int* status, int V, float* red, RowProj proj) {
    const int w = threadIdx.x >> 5;
    const bool want_traj = traj && t_iter < kTrajLen;
    const int nq = (n_pad + 31) >> 5;
    int r = 0;
    float b[8];
    if (w == 0) {  // the restart row, loaded while the split sums run
        r = act_idx ? __ldcg(act_idx + j) : j;
        load_row(B32, ldb, r, nq, n, b);
    }
    row_partials(part_acc, part_mom, splits, part_rows, n_pad, j, want_traj, V, NW, w, red);
    __syncthreads();
    if (w != 0) return;
    float accv[8], e2, e4;
    row_combine(red, V, n_pad, n, want_traj, accv, &e2, &e4);
    finish_row_loaded(accv, b, nq, n, r, j, B32, ldb, inv_T, tol, flags, iters, traj, t_iter, want_traj, e2, e4,
                      status, proj);
}
template <int NW>
__global__ void __launch_bounds__(NW * 32) finalize_kernel(const float* __restrict__ part_acc,
                                                           const float* __restrict__ part_mom, int splits,
                                                           int part_rows, int n_pad, int n,
                                                           const int* __restrict__ act_idx,
                                                           const int* __restrict__ count_dev, int M_act_host,
                                                           float* __restrict__ B32, int ldb, float inv_T, float tol,
                                                           int* __restrict__ flags, int* __restrict__ iters,
                                                           float* __restrict__ traj, int t_iter, int* status,
                                                           int* __restrict__ act_out, int* count_out,
                                                           long long* rows_accum, unsigned int* done_ctr,
                                                           const int* __restrict__ shape_dev, int vw_ctas,
                                                           RowProj proj) {
    extern __shared__ float fin_red[];  // [V][n_pad] sums, [V][n_pad] compensations, [V][4] moments
    pdl_wait();  // the update grid wrote the partials and the shape
    pdl_trigger();
    if (shape_dev) {  // split count and partial-row stride chosen on the device by the fused launch
        splits = shape_dev[0];
        part_rows = shape_dev[1];
    }
    const int M_act = count_dev ? *count_dev : M_act_host;
    const int j = blockIdx.x;
    if (j >= M_act) {  // the grid covers an upper bound of the active count
        if (j == 0 && threadIdx.x == 0) *count_out = 0;  // nothing active: empty list
        return;
    }
    // summation order: NW virtual warps, or (update loop of the BF16 stage) the persistent stage
    // kernel's order for this active count, so that both give identical rows
    const int V = vw_ctas > 0 ? fin_vwarps(M_act, vw_ctas) : NW;
    finalize_row<NW>(part_acc, part_mom, splits, part_rows, n_pad, n, act_idx, j, B32, ldb, inv_T, tol, flags, iters,
                     traj, t_iter, status, V, fin_red, proj);
    compact_tail<NW>(flags, act_idx, M_act, act_out, count_out, rows_accum, done_ctr, M_act);
}

// Rows with many splits and few rows (the refinement) get 32 warps each, others 4: with 8 warps
// (58 registers) only four blocks fit an SM and 1024 rows took 1.7 waves (ncu); one warp per
// row, even with four loads in flight per lane, was slower (too few warps to hide L2 latency).
cudaError_t launch_finalize(cudaStream_t s, const float* part_acc, const float* part_mom, int splits,
                            int part_rows, int n_pad, int n, const int* act_idx, const int* count_dev, int M_act,
                            float* B32, int ldb, double inv_T, double tol, int* flags, int* iters, float* traj,
                            int t_iter, int* status, int* act_out, int* count_out, long long* rows_accum,
                            unsigned int* done_ctr, const int* shape_dev, bool pdl, int vw_ctas, const float* Wp,
                            int nw, int ldw) {
    const float fT = static_cast<float>(inv_T), ftol = static_cast<float>(tol);
    const RowProj proj{Wp, Wp ? nw : 0, ldw};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(M_act, 1, 1);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (M_act <= 64 && splits > 16) {
        cudaError_t e = allow_max_dyn_smem(finalize_kernel<32>);
        if (e != cudaSuccess) return e;
        cfg.blockDim = dim3(1024, 1, 1);
        cfg.dynamicSmemBytes = sizeof(float) * 32 * (2 * n_pad + 4);
        return cudaLaunchKernelEx(&cfg, finalize_kernel<32>, part_acc, part_mom, splits, part_rows, n_pad, n, act_idx,
                                  count_dev, M_act, B32, ldb, fT, ftol, flags, iters, traj, t_iter, status, act_out,
                                  count_out, rows_accum, done_ctr, shape_dev, 0, proj);
    }
    cfg.blockDim = dim3(128, 1, 1);
    cfg.dynamicSmemBytes = sizeof(float) * (vw_ctas > 0 ? kFinMaxVWarps : 4) * (2 * n_pad + 4);
    return cudaLaunchKernelEx(&cfg, finalize_kernel<4>, part_acc, part_mom, splits, part_rows, n_pad, n, act_idx,
                              count_dev, M_act, B32, ldb, fT, ftol, flags, iters, traj, t_iter, status, act_out,
                              count_out, rows_accum, done_ctr, shape_dev, vw_ctas, proj);
}

// Un-normalised update (step entry point): Bnew = acc / T - 3 B and moments / T.
__global__ void combine_kernel(const float* __restrict__ part_acc, const float* __restrict__ part_mom, int splits,
                               int part_rows, int n_pad, int M, const float* __restrict__ B, double inv_T,
                               float* __restrict__ Bnew, float* __restrict__ moments) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < static_cast<int64_t>(M) * n_pad) {
        const int row = static_cast<int>(i / n_pad), k = static_cast<int>(i % n_pad);
        double acc = 0.0;
        for (int sp = 0; sp < splits; ++sp)
            acc += static_cast<double>(part_acc[(static_cast<int64_t>(sp) * part_rows + row) * n_pad + k]);
        Bnew[i] = static_cast<float>(acc * inv_T - 3.0 * static_cast<double>(B[i]));
    }
    if (moments && i < static_cast<int64_t>(M) * 4) {
        const int row = static_cast<int>(i / 4), c = static_cast<int>(i % 4);
        double acc = 0.0;
        if (c < 3)
            for (int sp = 0; sp < splits; ++sp)
                acc += static_cast<double>(part_mom[(static_cast<int64_t>(sp) * part_rows + row) * 4 + c]);
        moments[i] = static_cast<float>(acc * inv_T);
    }
}

cudaError_t launch_combine(cudaStream_t s, const float* part_acc, const float* part_mom, int splits, int part_rows,
                           int n_pad, int M, const float* B, double inv_T, float* Bnew, float* moments) {
    const int64_t total = static_cast<int64_t>(M) * (n_pad > 4 ? n_pad : 4);
    combine_kernel<<<static_cast<int>((total + 255) / 256), 256, 0, s>>>(part_acc, part_mom, splits, part_rows,
                                                                          n_pad, M, B, inv_T, Bnew, moments);
    return cudaGetLastError();
}

// Valid entries (>= 0) of the candidate slots, in order, to two lists and a device count.
__global__ void compact_cand_kernel(const int* cand, int k, int* list_a, int* list_b, int* count_dev) {
    if (threadIdx.x != 0) return;
    int c = 0;
    for (int j = 0; j < k; ++j)
        if (cand[j] >= 0) {
            list_a[c] = cand[j];
            list_b[c] = cand[j];
            ++c;
        }
    *count_dev = c;
}
cudaError_t launch_compact_cand(cudaStream_t s, const int* cand, int k, int* list_a, int* list_b, int* count_dev) {
    compact_cand_kernel<<<1, 32, 0, s>>>(cand, k, list_a, list_b, count_dev);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Kurtosis and objective of candidate rows from split-T moment partials (Eq. 2, Eq. 1).
// m2 = mean z^2, m4 = mean z^4, q = mean (z^2 - 1)^2. alpha + 2 = m4/m2^2 - 1 is formed as
// (q - (m2 - 1)^2) / m2^2, which has no cancellation when z^2 ~ 1 (binary-like components
// whose alpha sits just above -2, where Upsilon is steep).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void alpha_upsilon(double m2, double m4, double q, double& alpha, double& ups) {
    const double a2 = (q - (m2 - 1.0) * (m2 - 1.0)) / (m2 * m2);
    alpha = a2 - 2.0;
    if (!(m2 > 0.0) || !isfinite(a2)) {
        alpha = 0.0;
        ups = -INFINITY;  // never selected
        return;
    }
    ups = a2 > 0.0 ? alpha - 2.0 * log(0.5 * a2) : INFINITY;
    (void)m4;
}

__global__ void kurt_finalize_kernel(const float* __restrict__ part_mom, int splits, int part_rows,
                                     const int* __restrict__ act_idx, const int* __restrict__ count_dev, int count_host,
                                     double inv_T, double* __restrict__ alpha, double* __restrict__ ups) {
    const int count = count_dev ? *count_dev : count_host;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    double m2 = 0.0, m4 = 0.0, q = 0.0;
    for (int sp = 0; sp < splits; ++sp) {
        const float* p = part_mom + (static_cast<int64_t>(sp) * part_rows + j) * 4;
        m2 += p[0];
        m4 += p[1];
        q += p[2];
    }
    double a, u;
    alpha_upsilon(m2 * inv_T, m4 * inv_T, q * inv_T, a, u);
    const int r = act_idx ? act_idx[j] : j;
    alpha[r] = a;
    ups[r] = u;
}

cudaError_t launch_kurt_finalize(cudaStream_t s, const float* part_mom, int splits, int part_rows,
                                 const int* act_idx, const int* count_dev, int count, double inv_T, double* alpha,
                                 double* ups) {
    kurt_finalize_kernel<<<(count + 255) / 256, 256, 0, s>>>(part_mom, splits, part_rows, act_idx, count_dev, count,
                                                              inv_T, alpha, ups);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Candidate selection: p = argmax Upsilon (Algorithm 2), ties to the lowest restart index.
// Distinct top-k: repeat {argmax over non-excluded rows; exclude every row whose direction
// matches the pick up to sign (|cos| >= threshold)}.
// ------------------------------------------------------------------------------------------
__global__ void select_clear_kernel(int* excluded, const int* init, int M, int* cand, int kmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) excluded[i] = init ? init[i] : 0;
    if (i < kmax) cand[i] = -1;
}
// Excluded mask := init (restarts dropped by the pruner) or zero; candidate slots := -1.
cudaError_t launch_select_clear(cudaStream_t s, int* excluded, const int* init, int M, int* cand, int kmax) {
    const int n = M > kmax ? M : kmax;
    select_clear_kernel<<<(n + 255) / 256, 256, 0, s>>>(excluded, init, M, cand, kmax);
    return cudaGetLastError();
}

// Stable compaction of the active list by keep flags (one CTA of 1024 threads, each owning a
// contiguous slice): used when the pruner drops restarts.
__global__ void __launch_bounds__(1024) compact_keep_kernel(const int* __restrict__ keep,
                                                            const int* __restrict__ act_in,
                                                            const int* __restrict__ count_in_dev, int count_host,
                                                            int* __restrict__ act_out, int* count_out_dev,
                                                            int invert) {
    __shared__ int warp_tot[32];
    const int count = count_in_dev ? *count_in_dev : count_host;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (count + 1023) / 1024;
    const int b = t * per, e = min(count, b + per);
    int local = 0;
    for (int i = b; i < e; ++i) local += (keep[i] != 0) != (invert != 0);
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
    for (int i = b; i < e; ++i)
        if ((keep[i] != 0) != (invert != 0)) act_out[pos++] = act_in ? act_in[i] : i;
    if (t == 1023) *count_out_dev = before + incl;
}
cudaError_t launch_compact_keep(cudaStream_t s, const int* keep, const int* act_in, const int* count_in_dev,
                                int count_host, int* act_out, int* count_out_dev, bool invert) {
    compact_keep_kernel<<<1, 1024, 0, s>>>(keep, act_in, count_in_dev, count_host, act_out, count_out_dev,
                                           invert ? 1 : 0);
    return cudaGetLastError();
}

__device__ __forceinline__ bool better(double u, int i, double bu, int bi) {
    if (bi < 0) return true;
    if (u > bu) return true;
    return u == bu && i < bi;
}

// subset == nullptr: candidates are rows 0..count-1; else rows subset[0..count) (entries < 0
// are skipped). Writes the winning row (or -1) to *out_slot.
__global__ void __launch_bounds__(1024) argmax_kernel(const double* __restrict__ ups, const int* __restrict__ excluded,
                                                      const int* __restrict__ subset, const int* __restrict__ count_dev,
                                                      int count_host, int* out_slot) {
    __shared__ double su[32];
    __shared__ int si[32];
    const int count = count_dev ? *count_dev : count_host;
    double bu = -INFINITY;
    int bi = -1;
    for (int j = threadIdx.x; j < count; j += blockDim.x) {
        const int r = subset ? subset[j] : j;
        if (r < 0) continue;
        if (excluded && excluded[r]) continue;
        const double u = ups[r];
        if (u != u || u == -INFINITY) continue;
        if (better(u, r, bu, bi)) {
            bu = u;
            bi = r;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ou = __shfl_xor_sync(0xffffffffu, bu, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && better(ou, oi, bu, bi)) {
            bu = ou;
            bi = oi;
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        su[w] = bu;
        si[w] = bi;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        bu = lane < nw ? su[lane] : -INFINITY;
        bi = lane < nw ? si[lane] : -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ou = __shfl_xor_sync(0xffffffffu, bu, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oi >= 0 && better(ou, oi, bu, bi)) {
                bu = ou;
                bi = oi;
            }
        }
        if (lane == 0) *out_slot = bi;
    }
}

cudaError_t launch_argmax(cudaStream_t s, const double* ups, const int* excluded, const int* subset,
                          const int* count_dev, int count, int* out_slot) {
    argmax_kernel<<<1, 1024, 0, s>>>(ups, excluded, subset, count_dev, count, out_slot);
    return cudaGetLastError();
}

// One warp per restart row: exclude it when |b . b_sel| >= cos_thresh (same optimum up to sign).
__global__ void exclude_kernel(const float* __restrict__ B32, int ldb, int n, int M, const int* sel_slot,
                               int* excluded, double cos_thresh) {
    const int sel = *sel_slot;
    if (sel < 0) return;
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= M) return;
    double dot = 0.0, na = 0.0, nb = 0.0;
    for (int k = lane; k < n; k += 32) {
        const double a = B32[static_cast<int64_t>(r) * ldb + k];
        const double b = B32[static_cast<int64_t>(sel) * ldb + k];
        dot += a * b;
        na += a * a;
        nb += b * b;
    }
    dot = warp_sum(dot);
    na = warp_sum(na);
    nb = warp_sum(nb);
    if (lane == 0 && (r == sel || fabs(dot) >= cos_thresh * sqrt(na * nb))) excluded[r] = 1;
}

cudaError_t launch_exclude(cudaStream_t s, const float* B32, int ldb, int n, int M, const int* sel_slot,
                           int* excluded, double cos_thresh) {
    exclude_kernel<<<(M * 32 + 255) / 256, 256, 0, s>>>(B32, ldb, n, M, sel_slot, excluded, cos_thresh);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Append (Algorithm 2, last step): w_i = b_p G (n-dim winner mapped back to N channels; Section
// 3.3), computed in FP64 after renormalising b_p. The rows of G are orthogonal to the earlier
// rows of W in exact arithmetic; in FP64 they are so only up to cond(F~F~^T) * eps, so w_i is
// re-orthogonalised against W[0..i) (classical Gram-Schmidt, applied twice) and renormalised,
// which keeps W W^T = I at rounding level. The sign is made canonical (largest-magnitude entry
// positive, first on ties). comp_stats receives (p, alpha_p, Upsilon_p).
// ------------------------------------------------------------------------------------------
__device__ double block_sum256(double v, double* red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    return s;
}

__global__ void __launch_bounds__(256) append_kernel(const double* __restrict__ G, int n, int N,
                                                     const float* __restrict__ B32, int ldb, const int* p_slot,
                                                     const double* __restrict__ alpha, const double* __restrict__ ups,
                                                     double* __restrict__ W, int i, double* kurt_out,
                                                     double* comp_stats) {
    __shared__ double b[kMaxN];
    __shared__ double w[kMaxN];
    __shared__ double coef[kMaxN];
    __shared__ double red[8];
    __shared__ int redi[8];
    const int p = *p_slot;
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    double* W_row = W + static_cast<int64_t>(i) * N;
    if (p < 0) {
        if (t < N) W_row[t] = 0.0;
        if (t == 0) {
            *kurt_out = 0.0;
            comp_stats[0] = -1.0;
        }
        return;
    }
    const double v = t < n ? static_cast<double>(B32[static_cast<int64_t>(p) * ldb + t]) : 0.0;
    const double ss = block_sum256(v * v, red);
    if (t < n) b[t] = v / sqrt(ss);
    __syncthreads();
    double acc = 0.0;
    if (t < N)
        for (int r = 0; r < n; ++r) acc += b[r] * G[static_cast<int64_t>(r) * N + t];
    if (t < N) w[t] = acc;
    __syncthreads();
    for (int pass = 0; pass < 2 && i > 0; ++pass) {
        // coef[j] = W_j . w (one thread per earlier row), then w -= sum_j coef[j] W_j
        for (int j = t; j < i; j += 256) {
            double d = 0.0;
            for (int c = 0; c < N; ++c) d += W[static_cast<int64_t>(j) * N + c] * w[c];
            coef[j] = d;
        }
        __syncthreads();
        if (t < N) {
            double x = w[t];
            for (int j = 0; j < i; ++j) x -= coef[j] * W[static_cast<int64_t>(j) * N + t];
            acc = x;
        }
        __syncthreads();
        if (t < N) w[t] = acc;
        __syncthreads();
    }
    const double nn = block_sum256(t < N ? acc * acc : 0.0, red);
    acc = t < N ? acc / sqrt(nn) : 0.0;
    // canonical sign: argmax |w| (lowest index on ties)
    double best = t < N ? fabs(acc) : -1.0;
    int bi = t < N ? t : 1 << 30;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    __syncthreads();
    if (lane == 0) {
        red[wp] = best;
        redi[wp] = bi;
    }
    __syncthreads();
    best = red[0];
    bi = redi[0];
    for (int k = 1; k < 8; ++k)
        if (red[k] > best || (red[k] == best && redi[k] < bi)) {
            best = red[k];
            bi = redi[k];
        }
    __syncthreads();
    if (t == bi) red[0] = acc;
    __syncthreads();
    const double sgn = red[0] < 0.0 ? -1.0 : 1.0;
    if (t < N) W_row[t] = sgn * acc;
    if (t == 0) {
        *kurt_out = alpha[p];
        comp_stats[0] = static_cast<double>(p);
        comp_stats[1] = alpha[p];
        comp_stats[2] = ups[p];
    }
}

cudaError_t launch_append(cudaStream_t s, const double* G, int n, int N, const float* B32, int ldb, const int* p_slot,
                          const double* alpha, const double* ups, double* W, int i, double* kurt_out,
                          double* comp_stats) {
    append_kernel<<<1, 256, 0, s>>>(G, n, N, B32, ldb, p_slot, alpha, ups, W, i, kurt_out, comp_stats);
    return cudaGetLastError();
}

// Algorithm 1 (FastICA with projection deflation, Section 2.2): initial restarts are random
// vectors in the full whitened space, projected onto the complement of the components found so
// far (w <- w - W^T (W w)) and normalised. One warp per row.
__global__ void __launch_bounds__(256) project_rows_kernel(float* __restrict__ B32, int ldb, int M, int n,
                                                           const float* __restrict__ W32, int nw, int ldw) {
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= M) return;
    float* b = B32 + static_cast<int64_t>(row) * ldb;
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k = lane + 32 * q;
        v[q] = k < n ? b[k] : 0.f;
    }
    for (int i = 0; i < nw; ++i) {
        const float* wi = W32 + static_cast<int64_t>(i) * ldw;
        float d = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = lane + 32 * q;
            if (k < n) d = fmaf(wi[k], v[q], d);
        }
        d = warp_sumf(d);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = lane + 32 * q;
            if (k < n) v[q] = fmaf(-d, wi[k], v[q]);
        }
    }
    float ss = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) ss = fmaf(v[q], v[q], ss);
    ss = warp_sumf(ss);
    const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k = lane + 32 * q;
        if (k < n) b[k] = v[q] * inv;
    }
}
cudaError_t launch_project_rows(cudaStream_t s, float* B32, int ldb, int M, int n, const float* W32, int nw, int ldw) {
    project_rows_kernel<<<(M + 7) / 8, 256, 0, s>>>(B32, ldb, M, n, W32, nw, ldw);
    return cudaGetLastError();
}

__global__ void w_to_f32_kernel(const double* __restrict__ W, int i, int N, float* __restrict__ W32, int ldw) {
    for (int k = threadIdx.x; k < ldw; k += blockDim.x)
        W32[static_cast<int64_t>(i) * ldw + k] = k < N ? static_cast<float>(W[static_cast<int64_t>(i) * N + k]) : 0.f;
}
cudaError_t launch_w_to_f32(cudaStream_t s, const double* W, int i, int N, float* W32, int ldw) {
    w_to_f32_kernel<<<1, 256, 0, s>>>(W, i, N, W32, ldw);
    return cudaGetLastError();
}

// Candidates of component i in the full whitened space (Section 3.3: w = G^T b), one block per
// slot j < k: the refined restart row b_r (r = cand[j]) normalised in FP64, w = G^T b normalised,
// written to out[j * N ..]; a zero row when the slot is empty (cand[j] < 0).
__global__ void __launch_bounds__(256) record_cands_kernel(const double* __restrict__ G, int n, int N,
                                                           const float* __restrict__ B32, int ldb,
                                                           const int* __restrict__ cand, double* __restrict__ out) {
    __shared__ double b[kMaxN];
    __shared__ double red[8];
    const int j = blockIdx.x, t = threadIdx.x;
    const int r = cand[j];
    double* row = out + static_cast<int64_t>(j) * N;
    if (r < 0) {
        if (t < N) row[t] = 0.0;
        return;
    }
    const double v = t < n ? static_cast<double>(B32[static_cast<int64_t>(r) * ldb + t]) : 0.0;
    const double ss = block_sum256(v * v, red);
    if (t < n) b[t] = v / sqrt(ss);
    __syncthreads();
    double acc = 0.0;
    if (t < N)
        for (int l = 0; l < n; ++l) acc += b[l] * G[static_cast<int64_t>(l) * N + t];
    const double nn = block_sum256(t < N ? acc * acc : 0.0, red);
    if (t < N) row[t] = acc / sqrt(nn);
}
cudaError_t launch_record_cands(cudaStream_t s, const double* G, int n, int N, const float* B32, int ldb,
                                const int* cand, int k, double* out) {
    record_cands_kernel<<<k, 256, 0, s>>>(G, n, N, B32, ldb, cand, out);
    return cudaGetLastError();
}

}  // namespace ica
