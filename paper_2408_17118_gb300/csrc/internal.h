// Internal launch interface between the translation units of the ordering-ICA library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace ica {

constexpr int kMaxN = 256;            // channels (and reduced dimension) supported
// Raises a kernel's dynamic shared memory limit to the largest the device allows (the opt-in
// per-block maximum minus the kernel's static shared memory). Kernels whose launches need
// different amounts always set this one value, so that host threads launching the same kernel
// concurrently with different sizes never race on the attribute.
template <typename F>
inline cudaError_t allow_max_dyn_smem(F* fn) {
    static const int optin = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        return v;
    }();
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(fn));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - static_cast<int>(a.sharedSizeBytes));
}
constexpr int kMaxCTAs = 4 * 152;     // cap on (split x restart-tile) CTAs of one fused launch
constexpr int kTrajLen = 5;           // iterations of per-restart features kept (pruner input)
constexpr int kFp32Rows = 64;         // restart rows per CTA, FP32 fused kernel
constexpr int kTcRows = 128;          // restart rows per CTA, tcgen05 fused kernel

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }
inline int64_t round_up64(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// ---- k_small.cu ----
cudaError_t launch_init_restarts(cudaStream_t s, uint64_t seed, int comp, int M, int n, int ldb,
                                 const float* B0, int B0_ld, float* B);
cudaError_t launch_iota(cudaStream_t s, int* idx, int count, int* count_dev);
cudaError_t launch_finalize(cudaStream_t s, const float* part_acc, const float* part_mom, int splits,
                            int part_rows, int n_pad, int n, const int* act_idx, const int* count_dev, int M_act,
                            float* B32, int ldb, double inv_T, double tol, int* flags, int* iters, float* traj,
                            int t_iter, int* status, int* act_out, int* count_out, long long* rows_accum,
                            unsigned int* done_ctr, const int* shape_dev = nullptr, bool pdl = false,
                            int vw_ctas = 0, const float* Wp = nullptr, int nw = 0, int ldw = 0);
// Order of the compensated sums over split partials in the BF16 stage's row completion: the
// number of virtual warps V per row (split s goes to virtual warp s mod V; the V sums are added
// in order). More virtual warps when few rows share the GPU, so that the persistent stage kernel
// finishes every row in one round of its CTAs' 16 warps (ctas = CTAs of the update). The
// per-launch finalize follows the same order when given vw_ctas, so both paths agree bit for bit.
constexpr int kFinMaxVWarps = 16;
__host__ __device__ inline int fin_vwarps(int M_act, int ctas) {
    return M_act <= ctas ? 16 : (M_act <= 4 * ctas ? 4 : 2);
}
cudaError_t launch_combine(cudaStream_t s, const float* part_acc, const float* part_mom, int splits,
                           int part_rows, int n_pad, int M, const float* B, double inv_T, float* Bnew,
                           float* moments);
cudaError_t launch_compact_cand(cudaStream_t s, const int* cand, int k, int* list_a, int* list_b, int* count_dev);
cudaError_t launch_kurt_finalize(cudaStream_t s, const float* part_mom, int splits, int part_rows,
                                 const int* act_idx, const int* count_dev, int count, double inv_T, double* alpha,
                                 double* ups);
cudaError_t launch_select_clear(cudaStream_t s, int* excluded, const int* init, int M, int* cand, int kmax);
cudaError_t launch_argmax(cudaStream_t s, const double* ups, const int* excluded, const int* subset,
                          const int* count_dev, int count, int* out_slot);
cudaError_t launch_exclude(cudaStream_t s, const float* B32, int ldb, int n, int M, const int* sel_slot,
                           int* excluded, double cos_thresh);
cudaError_t launch_append(cudaStream_t s, const double* G, int n, int N, const float* B32, int ldb,
                          const int* p_slot, const double* alpha, const double* ups, double* W, int i,
                          double* kurt_out, double* comp_stats);
// Algorithm 1 helpers: rows of B (M x ldb, first n entries) projected onto the complement of the
// nw FP32 rows of W32 (ld ldw) and normalised; row i of the FP64 W (ld N) converted to FP32 (ld ldw).
cudaError_t launch_project_rows(cudaStream_t s, float* B32, int ldb, int M, int n, const float* W32, int nw, int ldw);
cudaError_t launch_w_to_f32(cudaStream_t s, const double* W, int i, int N, float* W32, int ldw);
cudaError_t launch_record_cands(cudaStream_t s, const double* G, int n, int N, const float* B32, int ldb,
                                const int* cand, int k, double* out);

// ---- k_linalg.cu ----
cudaError_t launch_row_mean(cudaStream_t s, const float* X, int N, int64_t T, int64_t ld, double* mean,
                            int* status = nullptr);
cudaError_t launch_covariance(cudaStream_t s, const float* X, const double* mean, int N, int64_t T,
                              int64_t ld, double* part, int splits, double* C);
int covariance_splits(int N, int64_t T);
// Symmetric eigendecomposition A = V diag(lam) V^T (cyclic Jacobi). scratch: device memory of
// jacobi_scratch_bytes(m) for the mixed-precision solver at m above its shared-memory limit
// (null: FP64 sweeps only there).
size_t jacobi_scratch_bytes(int m);
cudaError_t launch_jacobi(cudaStream_t s, double* A, double* V, double* lam, int m, int* status,
                          int max_sweeps, void* scratch = nullptr);
cudaError_t launch_gemm_f64(cudaStream_t s, int rows, int cols, int inner, double alpha, const double* A,
                            int64_t sar, int64_t sac, const double* B, int64_t sbr, int64_t sbc, double beta,
                            double* C, int64_t ldc);
cudaError_t launch_set_identity(cudaStream_t s, double* A, int rows, int cols, int64_t ld, double diag);
cudaError_t launch_scale_cols_fn(cudaStream_t s, const double* Q, const double* lam, int m, int fn,
                                 double* out, int* status, double ill_thresh);
cudaError_t launch_axpby_f64(cudaStream_t s, int64_t n, double a, const double* x, double b,
                             const double* y, double* out);
cudaError_t launch_pad_cols(cudaStream_t s, const double* W, int k, int N, int ncols, double* out);

// ---- k_reduce.cu ----
cudaError_t launch_rows_gemm(cudaStream_t s, const double* G, int n, int n_pad, int N, const float* X,
                             int64_t T, int64_t ldxin, const double* bias, float* out32, int64_t ld32,
                             uint16_t* out16, int64_t ld16);
// E4M3 copy of the FP32 rows X32 (n rows of ldx floats; rows n..n8-1 and samples T..ld8-1 zero) into
// X8 (n8 rows of ld8 bytes, ld8 a multiple of 16, n8 <= 256), row k scaled by a power of two 2^e_k
// that maps its largest magnitude into [-448, 448]. sc (3 n8 + 1 floats): 2^e_k, 2^(c - e_k),
// 2^-e_k and 2^-c with c = 8 + min_k e_k. rmax: n8 unsigned scratch. *launches += kernels launched.
cudaError_t launch_fp8_copy(cudaStream_t s, const float* X32, int64_t ldx, int64_t T, int n, int n8,
                            unsigned* rmax, float* sc, uint8_t* X8, int64_t ld8, int* launches);

// ---- k_fp32.cu ----
size_t fp32_smem_bytes(int n_pad);
cudaError_t launch_fused_fp32(cudaStream_t s, bool moments_only, const float* B32, int ldb,
                              const int* act_idx, const int* count_dev, int M_act, const float* Xt, int64_t ldx,
                              int n_pad, int64_t T, int splits, int chunks_per_split, float* part_acc,
                              float* part_mom, int part_rows);
constexpr int kFp32SmallRows = 16;  // at most this many rows go to the few-row FP32 kernel
int fp32_rows_tile(int M_act);       // its row tile (4 or 16) for M_act <= kFp32SmallRows rows
int fp32_rows_chunk(int n_pad);      // samples per chunk of the few-row kernel
size_t fp32_rows_smem_bytes(int n_pad, int R);
cudaError_t launch_fused_fp32_rows(cudaStream_t s, bool moments_only, const float* B32, int ldb, const int* act_idx,
                                   const int* count_dev, int M_act_host, const float* Xt, int64_t ldx, int n_pad,
                                   int64_t T, int splits, int chunks_per_split, float* part_acc, float* part_mom,
                                   int part_rows, bool pdl = false);

// ---- k_mlp.cu (learned restart pruner) ----
constexpr int kMlpIn = 13, kMlpHid = 64;
constexpr int kMlpParams = 2 * kMlpIn + kMlpHid * kMlpIn + kMlpHid + kMlpHid * kMlpHid + kMlpHid + kMlpHid + 1;
constexpr int kActRow = 272;  // floats of training activations per sample
int mlp_slices(int rows);
size_t mlp_scratch_bytes(int rows);
cudaError_t launch_mlp_init(cudaStream_t s, uint64_t seed, float* params);
cudaError_t launch_mlp_standardize(cudaStream_t s, const float* F, int rows, float* params);
cudaError_t launch_mlp_forward(cudaStream_t s, const float* params, const float* F, int rows, bool fp16, float* prob);
cudaError_t launch_mlp_train_step(cudaStream_t s, float* params, float* m, float* v, int step, const float* F,
                                  const float* y, int rows, float lr, float pos_weight, bool fp16, float* scratch,
                                  float* loss_out, float* grad_out);
// Keep set of the pruner after iteration kTrajLen: the network's keeps (p >= tau), minus the
// restarts dominated by a similar (|cos| >= cos_min; 0 disables) restart leading them in
// Upsilon, plus the keep floor: the max(keep_min, ceil(keep_frac * count)) restarts with the
// largest Upsilon at iteration kTrajLen (and any tied with the last of them).
// gauss_thr > 0: when no running restart's Upsilon reaches it (the Gaussianity threshold of
// Eq. 3), the network keeps nothing and only the keep floor stays.
cudaError_t launch_prune(cudaStream_t s, const float* params, const float* traj, const int* act_idx,
                         const int* count_dev, int count_host, int n, double logT, float tau, float gauss_thr,
                         float* ref, int* keep, int* pruned, int keep_min, float keep_frac, const float* B32, int ldb,
                         int row_n, float cos_min, int* order);  // order: scratch of count ints (sorted test)
cudaError_t launch_record(cudaStream_t s, const float* traj, const int* iters, const float* B32, int ldb, int n, int M,
                          const int* slot, double logT, float* ref, float* F_out, float* y_out);
// 1 in *out when some pruned restart's Upsilon at iteration kTrajLen (its objective when it was
// pruned) is at least the best final Upsilon of the restarts that stayed.
cudaError_t launch_prune_check(cudaStream_t s, const double* ups, const int* pruned, const float* traj, int M,
                               int* out);
// Stable compaction of an index list (act_in, or 0..count-1) to the slots whose keep flag is set
// (invert: whose flag is clear).
cudaError_t launch_compact_keep(cudaStream_t s, const int* keep, const int* act_in, const int* count_in_dev,
                                int count_host, int* act_out, int* count_out_dev, bool invert = false);

// Launch shape of a fused tcgen05 update from the device count of active rows (also evaluated
// by the finalize): tiles of 128 rows, splits of the sample range so that tiles x splits <= ctas
// (one wave), chunks per split.
__host__ __device__ inline void tc_device_shape(int M_act, int ctas, int total_chunks, int* tiles, int* splits,
                                                int* cps) {
    const int t = (M_act + kTcRows - 1) / kTcRows;
    int s = t < 1 ? 1 : (t <= ctas ? ctas / t : 1);
    if (s > total_chunks) s = total_chunks;
    if (s < 1) s = 1;
    const int c = (total_chunks + s - 1) / s;
    *tiles = t;
    *cps = c;
    *splits = (total_chunks + c - 1) / c;
}
// ---- k_tc.cu ----
int tc_chunk(int n_pad);
int tc_buffers(int n_pad);
size_t tc_smem_bytes(int n_pad, bool moments_only, int* stages_out);
// xmap: X~ (n_pad x T, samples contiguous), box {64, n_pad}.
// use_lo = false: the restart rows enter the first product as one BF16 term (their high term).
cudaError_t launch_fused_tc_shaped(cudaStream_t s, bool moments, const CUtensorMap& xmap, const float* B32, int ldb,
                                   const int* act_idx, const int* count_dev, int M_ub, int n_pad, int64_t T, int ctas,
                                   int total_chunks, float* part_acc, float* part_mom, int* status, int* shape_out,
                                   bool use_lo = true);
cudaError_t launch_fused_tc(cudaStream_t s, bool moments_only, bool moments, const CUtensorMap& xmap,
                            const float* B32, int ldb, const int* act_idx,
                            const int* count_dev, int M_act, int n_pad, int64_t T, int splits, int chunks_per_split,
                            int total_chunks, float* part_acc, float* part_mom, int part_rows, int* status);

// ---- k_stage.cu ----
// Persistent BF16 stage: iterations [t_begin, t_end) of the update loop of one component in one
// cooperative launch of `ctas` CTAs (one per SM). The active list act_{cur0} / count_{cur0} is
// the input; ctl receives {iteration index reached, final active count, final list index}, and
// the final count is also stored in count_{ctl[2]}. bar_ctr must be zero. Returns
// cudaErrorCooperativeLaunchTooLarge, launching nothing, when the CTAs cannot all be resident.
struct StageLaunch {
    float* B32;
    int ldb;
    int *act0, *act1, *count0, *count1;
    int cur0;
    int n_pad, n;
    int64_t T;
    int ctas;
    float* part_acc;
    float* part_mom;
    int* flags;
    int* iters;
    float* traj;
    int* status;
    long long* rows_accum;
    unsigned int* bar_ctr;
    int* ctl;
    int t_begin, t_end;
    double inv_T, tol;
    uint64_t wait_ns;  // limit of the kernel's waits (0: ICA_WAIT_NS); its teardown drains keep ICA_WAIT_NS
    int stall;         // test hook: 1 makes the first grid barrier wait for an arrival that never comes
    const float* Wp;   // Algorithm 1: found components (nw rows, ld ldw, FP32) projected out of each update
    int nw, ldw;
    int lo_from;       // iterations t >= lo_from add the restart rows' low BF16 term (0: every iteration)
    int streamk;       // 1: equal shares of the (tile x chunk) work when the one-wave shape leaves SMs idle
    bool fp8;          // the FP8 form: E4M3 operands (xmap: the E4M3 copy of X~, box {128, round_up(n, 32)})
    float* zmax;       // per restart: largest |z| of its last update (null: not recorded)
    int track_until;   // iterations t with t + 1 < track_until record zmax (when zmax is set)
    const float* fp8sc; // FP8 form: scales of launch_fp8_copy
};
// resident (optional) receives the number of CTAs of the kernel that fit the GPU at once.
cudaError_t launch_stage_tc(cudaStream_t s, const CUtensorMap& xmap, const StageLaunch& p, int* resident = nullptr);

// ---- k_fp32.cu: persistent FP32 refinement ----
// Iterations [t_begin, t_end) of the refinement of at most rows_max (<= 4) candidate rows in one
// cooperative launch of `splits` CTAs (the per-launch loop's split of the sample range into
// chunks of fp32_rows_chunk(n_pad) samples, cps chunks per split). act_{cur0} / count_{cur0}
// hold the rows; ctl receives {iteration index reached, final count, final list index}; the
// final count is also stored in count_{ctl[2]}. bar_ctr must be zero. part_acc / part_mom need
// splits x 4 rows. Returns cudaErrorCooperativeLaunchTooLarge, launching nothing, when the CTAs
// cannot all be resident.
struct RefineLaunch {
    float* B32;
    int ldb;
    int *act0, *act1, *count0, *count1;
    int cur0;
    const float* Xt;
    int64_t ldx;
    int n_pad, n;
    int64_t T;
    int splits, cps, rows_max;
    float* part_acc;
    float* part_mom;
    int* flags;
    int* iters;
    int* status;
    long long* rows_accum;
    unsigned int* bar_ctr;
    int* ctl;
    int t_begin, t_end;
    float inv_T, tol;
    uint64_t wait_ns;  // limit of the grid barriers (0: ICA_WAIT_NS)
    const float* Wp;   // Algorithm 1: found components (nw rows, ld ldw, FP32) projected out of each update
    int nw, ldw;
};
cudaError_t launch_refine_fp32(cudaStream_t s, const RefineLaunch& p, int* resident = nullptr);

// ---- k_plain.cu ----
cudaError_t launch_gather_rows(cudaStream_t s, const float* B32, int ldb, const int* act_idx,
                               const int* count_dev, int M_act, int n_pad, float* out);
cudaError_t launch_cube_inplace(cudaStream_t s, float* Z, int rows, int64_t T, int64_t ldz);
cudaError_t launch_row_moments(cudaStream_t s, const float* Z, int rows, int64_t T, int64_t ldz,
                               float* part_mom);

}  // namespace ica
