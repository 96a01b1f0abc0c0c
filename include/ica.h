/*
 * ordering-ica GB300 library: C ABI.
 *
 * Batched kurtosis fixed-point iteration of the ordering ICA in matrix form (Matsuda &
 * Yamaguchi, "Efficient Estimation of Unique Components in Independent Component Analysis
 * by Matrix Representation", arXiv 2408.17118), on one NVIDIA GB300 (sm_103a).
 *
 * Conventions for every entry point:
 *   - Matrices are row-major. X and its derived data are N x T with the sample index T
 *     contiguous; "ld" arguments are row strides in elements.
 *   - Every array argument is a DEVICE pointer unless a comment says "host".
 *   - The caller owns every buffer, including the workspace (ica_set_workspace). After the
 *     workspace is set the library allocates no device memory (the optional plain FP32
 *     comparator creates a cuBLAS handle on first use, which allocates inside cuBLAS).
 *   - Work is enqueued on the context's stream (ica_set_stream). ica_order_fit synchronises
 *     that stream a few times per component: once after each persistent BF16 stage and FP32
 *     refinement launch (opts.stage_persistent), otherwise on a sparse schedule of iterations
 *     (it reads the active-restart count every fourth iteration on the BF16 path; every
 *     iteration at first, then every second and every fourth on the FP32 path; with the
 *     restart pruner also when it runs and before the kurtosis pass); ica_whiten,
 *     ica_deflation_basis, ica_fp_step and ica_kurtosis synchronise once at the end to read
 *     the device status word; ica_init_restarts, ica_reduce and ica_quantize_e4m3 only enqueue.
 *   - The return value is an ica_status. Nothing is thrown across the ABI. After an error the
 *     outputs are unspecified and the context stays usable.
 *   - The paper writes samples as M and restarts as L; this interface writes samples as T
 *     and restarts as M.
 */
#ifndef ORDERING_ICA_H
#define ORDERING_ICA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ica_ctx ica_ctx;

typedef enum {
    ICA_OK = 0,
    ICA_ERR_ARG = 1,          /* argument outside the documented range */
    ICA_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed */
    ICA_ERR_NONFINITE = 3,    /* a restart row became NaN/Inf or zero, or every restart died */
    ICA_ERR_ILLCOND = 4,      /* covariance or F~F~^T (Section 3.3) is numerically singular */
    ICA_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out (kernel returned early) */
    ICA_ERR_WORKSPACE = 6,    /* no workspace set, or smaller than ica_workspace_bytes() */
    ICA_ERR_UNSUPPORTED = 7   /* precision or feature not available (e.g. no cuBLAS) */
} ica_status;

typedef enum {
    ICA_FP32 = 0,        /* fused FP32 CUDA-core iteration (Z never stored) */
    ICA_BF16 = 1,        /* fused tcgen05 iteration, BF16 operands, FP32 accumulate and cube,
                            followed by FP32 refinement of the top distinct candidates */
    ICA_FP8 = 2,         /* as ICA_BF16, with iterations 1..fp8_iters of each component's stage
                            on E4M3 operands (tcgen05 kind::f8f6f4, FP32 accumulate and cube):
                            X~ with one power-of-two scale per row, the restart rows with a
                            power-of-two scale per column of X~, P = Z o Z o Z with one
                            power-of-two scale per restart row set from the row's largest |z| of
                            the previous iteration (Section 3.1's update, same fixed points; the
                            later BF16 iterations and the FP32 refinement set the accuracy). The
                            FP8 iterations need the persistent stage; otherwise they run in BF16. */
    ICA_PLAIN_FP32 = 3   /* Algorithm 2 written literally: Z = B X~ materialised in device
                            memory, cube, second product (cuBLAS SGEMM, no TF32). The
                            comparison baseline, not the fast path. */
} ica_precision;

/* Options of ica_order_fit. Fill with ica_default_opts, then override fields. */
typedef struct {
    int precision;         /* ica_precision (default ICA_BF16) */
    int gauss_test;        /* 1: stop when Upsilon(alpha_i) < 2(N-i+2)(N-i+1)/T (Eq. 3) */
    int refine_topk;       /* BF16: distinct candidates refined in FP32 per component (>= 1) */
    int refine_iters;      /* BF16: maximum FP32 refinement iterations (default 10: from a
                              BF16-converged start a non-Gaussian optimum converges in a few
                              cubically convergent steps; candidates still moving after 10 lie
                              in a near-Gaussian, flat part of the objective) */
    double stage_tol;      /* BF16: convergence tolerance of the BF16 stage */
    double refine_tol;     /* BF16: convergence tolerance of the FP32 refinement */
    double fp32_tol_floor; /* FP32 stages never use a tolerance below this (FP32 rounding) */
    const float* B0;       /* optional: n_components x M x N initial restarts (device, FP32);
                              component i uses the first N-i entries of each row (all N with
                              algorithm 1). NULL: draw
                              them from Philox4x32-10 keyed by the seed (ica_init_restarts). */
    int max_splits;        /* 0: automatic split of the sample range; >0 caps it (tests) */
    int profile;           /* 1: time every fused launch with CUDA events on the context stream
                              and report per-kind totals (launches, ms, algorithmic FLOPs) in
                              ica_last_stats */
    /* Learned restart pruner (not part of the paper's method; see ica_mlp_* below). */
    const float* prune_params; /* optional: ICA_MLP_PARAMS floats (device). After the first 5
                              iterations of a component, restarts whose predicted probability of
                              ending at the picked direction is below prune_tau leave the active
                              set and the pick (and so do restarts redundant with a leading
                              one, prune_cos), except the restarts leading the objective then:
                              the max(refine_topk (1 on the FP32 path), ceil(prune_keep_frac x
                              active)) restarts with the largest Upsilon (Eq. 1) at iteration 5
                              always stay. If a pruned restart's kurtosis objective is at
                              least the best kept one, or the pruner dropped every active
                              restart, the component is fitted again without pruning from the
                              same initial restarts (reported as "fallback" in ica_last_stats).
                              NULL: no pruning. Ignored by ICA_PLAIN_FP32. */
    float prune_tau;       /* keep-probability threshold (default 0.05) */
    float* record_features; /* optional (device): n_components x M x ICA_MLP_IN raw pruner inputs
                              of every restart (alpha at iterations 1..5, step distance at 1..5,
                              n = N - i + 1, log T, Upsilon gap at iteration 5), for training */
    float* record_labels;  /* optional (device, with record_features): n_components x M labels,
                              1 when the restart ended at the picked direction
                              (|b_r . b_p| >= 1 - 1e-3), else 0 */
    int stage_persistent;  /* BF16: 1 (default) runs each component's BF16 iterations as one
                              persistent cooperative launch (one CTA per SM, grid barriers
                              between the update, the row completion and the removal of
                              converged rows) when the fit has the GPU to itself (not inside a
                              multi-worker ica_order_fit_batched) and M <= 152 * 128; 0 launches
                              the update and the row completion per iteration. Both give the
                              same results. */
    int64_t wait_ns;       /* limit (ns) of every bounded wait of the persistent stage and
                              refinement kernels (mbarrier waits, grid barriers); 0: 2 s. When it
                              runs out the kernel stops, frees its resources and returns, and the
                              call reports ICA_ERR_TIMEOUT. The per-launch kernels and every
                              teardown drain keep the 2 s limit. */
    int stall_test;        /* test hook, 0 in normal use: 1 makes the first grid barrier of the
                              persistent stage wait for one arrival more than there are CTAs, so
                              that its wait runs out (exercises the timeout path on the host's
                              request, without a fault) */
    float prune_keep_frac; /* fraction of the active restarts, ranked by Upsilon at iteration 5,
                              that the pruner always keeps (default 0.05; 0..1; 0: no floor at
                              all) */
    float prune_cos;       /* the pruner also drops a restart when another one leading it in
                              Upsilon at iteration 5 points the same way, |b . b'| >= prune_cos
                              (it is heading to the same optimum); default 0.99, 0 disables.
                              The keep floor (prune_keep_frac) overrides it. */
    int prune_gauss;       /* pruner: 1 (default) - when no running restart's Upsilon at iteration 5
                              reaches the Gaussianity threshold of Eq. 3 for the component, the
                              component is in the Gaussian subspace (no unique direction,
                              Theorem 1) and only the keep floor stays; 0: the network decides */
    int algorithm;         /* 2 (default): Algorithm 2, each component on the reduced data X~ = G Xw
                              (Section 3.3, n = N - i + 1 dimensions). 1: Algorithm 1's form (the
                              "threads" ordering ICA, run here as one batch): every iteration on
                              the full whitened data (n = N), each update projected onto the
                              complement of the found components, w <- w - W^T (W w); the initial
                              restarts are N-dimensional (B0 rows use all N entries) and projected
                              the same way. Same fixed points, (N / n) times the work per
                              iteration (the comparison variant of Section 4). */
    int stage_lo_from;     /* BF16 stage: iterations t >= stage_lo_from (0-based) feed the restart
                              rows to the first product as two BF16 terms (hi + lo, about 16
                              bits: rows can converge to stage_tol); earlier ones as one BF16
                              term, which is enough far from convergence (default 5: the
                              iterations before the restart pruner's decision) */
    int stage_streamk;     /* persistent BF16 stage: 1 (default) - when the one-wave shape (restart
                              tiles x sample splits) would leave more than a sixteenth of the SMs
                              idle, every CTA takes an equal share of the (tile x chunk) work
                              instead (results then differ from the per-launch path by FP32
                              summation order); 0: always the one-wave shape */
    double* record_cands;  /* optional (device, BF16 / FP8 path): n_components x refine_topk x N
                              FP64. Row (i, j) = w = G^T b of the j-th distinct candidate of
                              component i after the FP32 refinement (Section 3.3: the candidate in
                              the full whitened space), normalised; zero rows where fewer
                              candidates were distinct. The pick of component i is among them. For
                              an FP64 re-check of the pick outside the library. */
    int fp8_iters;         /* ICA_FP8: stage iterations 1..fp8_iters (0-based) on E4M3 operands
                              (default 3, so that iteration 4, the last before the pruner, is BF16
                              again; 0: none) */
} ica_opts;

/* Default options: BF16, no Gaussianity test, refine_topk 4, refine_iters 10,
   stage_tol 1e-4, refine_tol 1e-6, fp32_tol_floor 1e-6, B0 NULL, automatic splits,
   no profiling, no pruner (prune_tau 0.05, prune_keep_frac 0.05, prune_cos 0.99), no
   recording, persistent stage, 2 s wait limit, no stall, algorithm 2, stage_lo_from 5,
   prune_gauss 1, stage_streamk 1, fp8_iters 3. */
void ica_default_opts(ica_opts* opts);

/* Human-readable name of a status code (static string). */
const char* ica_status_string(int status);

/* Text of the last CUDA runtime failure behind an ICA_ERR_CUDA returned to the calling host
   thread (the failing call and its error string); empty if none. Valid until the next call of
   this library from the same thread. */
const char* ica_last_error(void);

/* Create a context bound to CUDA device `device` (host pointer *out receives it). Allocates a
   small pinned host buffer for device->host counters. ICA_ERR_CUDA if the device is absent. */
int ica_create(ica_ctx** out, int device);

/* Destroy a context created by ica_create (NULL is accepted). Does not free caller buffers. */
int ica_destroy(ica_ctx* ctx);

/* Enqueue all further work on `stream` (a cudaStream_t; NULL = legacy default stream). */
int ica_set_stream(ica_ctx* ctx, void* stream);

/* Bytes of device workspace ica_order_fit needs for these sizes and options (also enough for
   every step entry point at the same or smaller sizes). Returns 0 for invalid sizes. */
size_t ica_workspace_bytes(int N, int64_t T, int M, const ica_opts* opts);

/* Hand the library a caller-allocated device workspace (256-byte aligned, `bytes` long). The
   library keeps the pointer until the next call or ica_destroy; it never frees it. */
int ica_set_workspace(ica_ctx* ctx, void* dev_ptr, size_t bytes);

/* Whitening ("X is whitened in advance", Section 2.2 and Theorem 1; symmetric form).
   X: N x T FP32 (ld = T). Outputs: Xw N x T FP32 (ld = T; must not alias X), V N x N FP64 and
   mean N FP64 with Xw = V (X - mean), V = C^(-1/2), C = (X - mean)(X - mean)^T / T. Means,
   covariance and the Jacobi eigendecomposition run in FP64 on the GPU.
   1 <= N <= 256, T >= 2N. ICA_ERR_ILLCOND if C has an eigenvalue <= 1e-12 * its largest. */
int ica_whiten(ica_ctx* ctx, const float* X, int N, int64_t T, float* Xw, double* V, double* mean);

/* Fast ordering ICA (Algorithm 2 with Section 3.1-3.3) on whitened Xw (N x T FP32, ld = T).
   For each component i = 1..n_components: reduction basis G (Eq. 6-7) and X~ = G Xw (Eq. 8);
   M restarts iterated in matrix form, Z = B X~, B <- (Z o Z o Z) X~^T / T - 3B, rows
   normalised, converged rows removed (min(||b-b_prev||, ||b+b_prev||) <= tol); kurtosis
   (Eq. 2) of every restart; p = argmax Upsilon (Eq. 1); w_i = b_p G appended.
   Outputs (device): W_out n_components x N FP64 (row i = component i, rows orthonormal, sign
   canonical: largest-magnitude entry positive), kurt_out n_components FP64 (alpha_i);
   n_found (HOST int) = components returned (< n_components only when gauss_test stops).
   1 <= N <= 256, T >= 2N, 1 <= M <= 65536, 1 <= n_components <= N, iters >= 1, tol > 0.
   Synchronises the context stream once per iteration. */
int ica_order_fit(ica_ctx* ctx, const float* Xw, int N, int64_t T, int M, int n_components,
                  int iters, double tol, uint64_t seed, const ica_opts* opts,
                  double* W_out, double* kurt_out, int* n_found);

/* Per-phase statistics of the last ica_order_fit as a JSON object written to the HOST buffer
   `buf` (NUL-terminated, at most `cap` bytes). Synchronises the context stream. */
int ica_last_stats(ica_ctx* ctx, char* buf, size_t cap);

/* ---------------------------------------------------------------------------------------
 * Step entry points: one hot-path step each, in the launch configuration ica_order_fit
 * uses. They need a workspace of ica_workspace_bytes(N or n, T, M, opts) at least.
 * --------------------------------------------------------------------------------------- */

/* Initial restarts of component `component` (Algorithm 2: random L x (N-i+1) matrix, rows
   normalised). Entry (l, 2j) / (l, 2j+1) come from one Philox4x32-10 call with counter
   (j, l, component, 0) and key (seed & 0xffffffff, seed >> 32): u = (k + 0.5) / 2^52 with
   k = (w_a >> 6) * 2^26 + (w_b >> 6) from words (0,1) and (2,3), Box-Muller in FP64, rows
   normalised in FP64. Output B: M x ldb FP32; columns n..ldb-1 are set to zero. */
int ica_init_restarts(ica_ctx* ctx, uint64_t seed, int component, int M, int n, float* B, int ldb);

/* Reduction basis (Section 3.3, Eq. 6-7): W k x N FP64 with orthonormal rows (ld = N),
   0 <= k < N. Output G: (N-k) x N FP64 (ld = N), G = (F~F~^T)^(-1/2) F~, F~ = first N-k rows
   of I - W^T W. ICA_ERR_ILLCOND if F~F~^T has an eigenvalue <= 1e-14. */
int ica_deflation_basis(ica_ctx* ctx, const double* W, int k, int N, double* G);

/* Reduction of signals (Eq. 8): X~ = G Xw. G: n x N FP64 (ld = N); Xw: N x T FP32 (ld = T).
   Outputs (either may be NULL): Xt32 n_pad x ldx32 FP32 and Xt16 n_pad x ldx16 BF16 (raw
   uint16 bits), n_pad = n rounded up to 16, rows n..n_pad-1 zero. ldx32, ldx16 >= T and
   multiples of 8. */
int ica_reduce(ica_ctx* ctx, const double* G, int n, int N, const float* Xw, int64_t T,
               float* Xt32, int64_t ldx32, uint16_t* Xt16, int64_t ldx16);

/* E4M3 operand of the FP8 iterations (ICA_FP8, Section 3.1's update on 8-bit operands): the
   FP32 reduced data Xt32 (n x ldx32, ld a multiple of 8) -> X8 (n8 rows of ld8 bytes, n8 = n
   rounded up to 32, ld8 >= T and a multiple of 16), row k stored as e4m3(x 2^e_k) (round to
   nearest even, saturating; byte 0x7e = 448), e_k the largest integer with max_t |x_kt| 2^e_k
   <= 448 (0 for a zero row); rows n..n8-1 and samples T..ld8-1 zero. scales (3 n8 + 1 floats):
   2^e_k, 2^(c - e_k) (the factor applied to column k of a restart row), 2^-e_k, and last 2^-c,
   c = 8 + min_{k<n} e_k. Needs a workspace of ica_workspace_bytes(n, T, 1, ICA_FP8 opts). */
int ica_quantize_e4m3(ica_ctx* ctx, const float* Xt32, int n, int64_t T, int64_t ldx32, uint8_t* X8, int64_t ld8,
                      float* scales);

/* One matrix-form update (Eq. 4-5 as written in Algorithm 2) for M rows without
   normalisation: Bnew = (Z o Z o Z) X~^T / T - 3 B with Z = B X~.
   precision ICA_FP32: Xt is FP32 n_pad x ldx; ICA_BF16: Xt is BF16 bits n_pad x ldx and B is
   rounded to BF16 for the products (FP32 accumulate, FP32 cube, BF16 cube operand).
   B, Bnew: M x n_pad FP32 (ld = n_pad, columns >= n ignored / written as the update of the
   zero padding, i.e. zero). moments (optional, M x 4 FP32): sum z^2 / T, sum z^4 / T. */
int ica_fp_step(ica_ctx* ctx, int precision, const float* B, int M, int n, const void* Xt,
                int64_t T, int64_t ldx, float* Bnew, float* moments);

/* Kurtosis and objective of M rows (Eq. 2 and Eq. 1; alpha normalised by the row's own
   second moment, alpha + 2 formed without cancellation):
   z = b X~, m2 = mean z^2, m4 = mean z^4, q = mean (z^2 - 1)^2,
   alpha = (q - (m2 - 1)^2) / m2^2 - 2, Upsilon = alpha - 2 log(alpha/2 + 1) (+inf if
   alpha <= -2). Precision and layouts as ica_fp_step. Outputs alpha, ups: M FP64. */
int ica_kurtosis(ica_ctx* ctx, int precision, const float* B, int M, int n, const void* Xt,
                 int64_t T, int64_t ldx, double* alpha, double* ups);

/* ---------------------------------------------------------------------------------------
 * Allocation-free entry point. (The paper has no counterpart: this is a deployment aid.)
 * --------------------------------------------------------------------------------------- */

/* Same computation and layouts as ica_fp_step, for callers that cannot call cudaMalloc at all:
   code inside an application whose allocator has already reserved the whole device (a
   framework caching allocator, an inference server's memory pool), plug-ins that may not
   allocate after start-up, or latency-critical loops that cannot afford cudaFree's implicit
   device synchronisation. It needs no context and no workspace: the split-T partial sums live
   in a 16 MiB array inside this library (one per GPU that loads the library, held until the
   process exits). It calls no cudaMalloc, cudaFree or other allocating routine.
   - Device: the call works on the CUDA device that is current on the calling host thread. B,
     Xt, Bnew, moments and the stream must belong to that device. The first call made with a
     given device current looks up that device's copy of the array (cudaGetSymbolAddress) and
     the tensor-map encoder.
   - Limit: M rows rounded up to the kernel's row tile (128 for ICA_BF16; 4 or 16 for ICA_FP32
     with M <= 16, else 64) times (round_up(n, 16) + 4) * 4 bytes must fit in 16 MiB less 256
     bytes, i.e. about 16,000 rows at n = 256; beyond it the call returns ICA_ERR_WORKSPACE
     without launching anything. Arguments outside ica_fp_step's range (M > 65536, ...) return
     ICA_ERR_ARG. The call runs the kernels ica_fp_step runs, with the same split of the sample
     range, so both give identical results, except when that split needs more than 16 MiB of
     partial sums: then it uses fewer pieces and results can differ from ica_fp_step's by FP32
     summation order.
   - Every call on a device shares the same array and the array keeps the last call's contents
     (the call clears the status word it needs zeroed). Calls whose kernels overlap on the GPU
     (different streams, or different host threads) race on it: serialise them.
   - stream: the cudaStream_t to enqueue on (NULL = legacy default stream). The call
     synchronises that stream at the end and copies the status word to host memory, so it must
     not be called while the stream is being captured into a CUDA graph. */
int ica_fp_step_noalloc(int precision, const float* B, int M, int n, const void* Xt, int64_t T,
                        int64_t ldx, float* Bnew, float* moments, void* stream);

/* ---------------------------------------------------------------------------------------
   Many data sets in one call. Not in the paper: the data sets of a batch (uneven N and T) are
   fitted concurrently by `workers` worker contexts, each with its own stream and a slice of the
   caller's workspace (set with ica_set_workspace, at least ica_batched_workspace_bytes). An
   autotuner times concurrent fused steps of the median data set for three GPU shares per
   launch (a full wave of CTAs, a half, a quarter) once per (workers, shape) and keeps the
   fastest. Data set k uses seed + k. The call returns after every fit finished; the caller's
   stream (ica_set_stream) is ordered before the first and after the last worker launch.
   opts->B0, record_features and record_labels must be NULL. ica_last_stats reports the
   batch (workers, chosen share, tuning times, wall time) and every data set's stats.
   --------------------------------------------------------------------------------------- */
typedef struct {
    const float* Xw;     /* whitened data, N x T row-major FP32 (device) */
    int N;               /* 1..256 */
    int64_t T;           /* >= 2N */
    int n_components;    /* 1..N */
    double* W_out;       /* n_components x N FP64 (device), as ica_order_fit */
    double* kurt_out;    /* n_components FP64 (device) */
    int* n_found;        /* host int */
} ica_dataset;

/* Workspace bytes for a batch (0 on invalid sizes); workers <= 0 means the default (8). */
size_t ica_batched_workspace_bytes(const ica_dataset* sets, int count, int M, const ica_opts* opts, int workers);

/* Fits every data set of the batch (Algorithm 2, as ica_order_fit, M restarts each). Returns
   the first non-OK status of any data set (outputs of the others are valid). */
int ica_order_fit_batched(ica_ctx* ctx, const ica_dataset* sets, int count, int M, int iters, double tol,
                          uint64_t seed, const ica_opts* opts, int workers);

/* ---------------------------------------------------------------------------------------
   Learned restart pruner: a 13-64-64-1 perceptron (ReLU, sigmoid output) trained on the
   trajectories the method itself records (record_features / record_labels above). Not part of
   the paper. Parameter vector layout (ICA_MLP_PARAMS FP32 values, device):
     mean[13], scale[13]        input standardisation x_hat = (x - mean) * scale
     W1[64][13], b1[64]         h1 = relu(W1 x_hat + b1)
     W2[64][64], b2[64]         h2 = relu(W2 h1 + b2)
     w3[64], b3                 p = sigmoid(w3 . h2 + b3)
   Feature rows (ICA_MLP_IN FP32 values): alpha at iterations 1..5, step distance at 1..5, n,
   log T, and Upsilon(alpha_5) (Eq. 1, alpha clamped at -1.999) minus the largest such value among
   the restarts still running at iteration 5. The kernels keep FP32 master weights; with fp16 = 1 weights and activations are
   rounded to FP16 (accumulation stays FP32), fp16 = 0 runs everything in FP32.
   --------------------------------------------------------------------------------------- */
#define ICA_MLP_IN 13
#define ICA_MLP_HIDDEN 64
#define ICA_MLP_PARAMS 5147

/* He-initialised weights (Philox4x32-10 keyed by seed), zero biases, mean 0, scale 1. */
int ica_mlp_init(ica_ctx* ctx, uint64_t seed, float* params);

/* Sets mean and scale of params from rows x ICA_MLP_IN feature rows F (population moments). */
int ica_mlp_standardize(ica_ctx* ctx, const float* F, int rows, float* params);

/* prob[r] = network output for feature row r (rows >= 1). Only enqueues. */
int ica_mlp_forward(ica_ctx* ctx, const float* params, const float* F, int rows, int fp16, float* prob);

/* Device scratch bytes ica_mlp_train_step needs for `rows` samples. */
size_t ica_mlp_scratch_bytes(int rows);

/* One full-batch training step on rows samples (labels 0/1): weighted binary cross-entropy
   L = -(1/rows) sum [pos_weight y log p + (1 - y) log(1 - p)], its gradient by
   back-propagation, then (lr > 0) one Adam update (beta 0.9, 0.999, eps 1e-8, bias-corrected
   with `step` >= 1) of every parameter except mean and scale. adam_m, adam_v: ICA_MLP_PARAMS
   floats each, zero before the first step. loss (1 float) and grad (ICA_MLP_PARAMS floats,
   mean and scale entries 0) are optional device outputs. scratch: caller-owned device memory of
   at least ica_mlp_scratch_bytes(rows). Deterministic (fixed reduction order). Only enqueues. */
int ica_mlp_train_step(ica_ctx* ctx, float* params, float* adam_m, float* adam_v, int step, const float* F,
                       const float* labels, int rows, float lr, float pos_weight, int fp16, void* scratch,
                       size_t scratch_bytes, float* loss, float* grad);

#ifdef __cplusplus
}
#endif

#endif /* ORDERING_ICA_H */
