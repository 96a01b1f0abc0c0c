// Host driver and C ABI of the ordering-ICA library. Implements Algorithm 2 (fast ordering ICA
// in matrix form, with removal of converged rows and reduction of signals) on one GPU:
// every arithmetic step runs in this library's kernels; the host only orders launches, picks
// launch shapes and reads back the active-restart count on a sparse schedule.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <dlfcn.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "ica.h"
#include "internal.h"

using namespace ica;

// ------------------------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------------------------
typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                      const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
typedef int (*PFN_cublasCreate_t)(void**);
typedef int (*PFN_cublasDestroy_t)(void*);
typedef int (*PFN_cublasSetStream_t)(void*, cudaStream_t);
typedef int (*PFN_cublasSgemm_t)(void*, int, int, int, int, int, const float*, const float*, int, const float*, int,
                                 const float*, float*, int);

struct ica_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint8_t* ws = nullptr;
    size_t ws_bytes = 0;
    int* host_i = nullptr;     // pinned: [0] count, [1] status, [2..65] candidate ids
    double* host_d = nullptr;  // pinned: component stats
    PFN_encodeTiled_t encode = nullptr;
    void* cublas_lib = nullptr;
    void* cublas = nullptr;
    PFN_cublasSgemm_t sgemm = nullptr;
    PFN_cublasSetStream_t cublas_set_stream = nullptr;
    PFN_cublasDestroy_t cublas_destroy = nullptr;
    std::string stats;
    // launch accounting and optional per-launch timing of the fused kernels
    long long launches = 0;        // kernels launched by the last ica_order_fit
    long long launches_total = 0;  // kernels launched by this context since ica_create
    std::vector<cudaEvent_t> ev;
    struct Rec {
        int kind;
        double flops;
        int e0, e1;
    };
    std::vector<Rec> recs;
    double kind_ms[10] = {}, kind_flops[10] = {};
    long long kind_n[10] = {};
    // share of the GPU (CTAs per launch, as a fraction of one wave) that fused launches aim
    // for: 1 when the fit owns the GPU, smaller when several fits run concurrently
    int cta_div = 1;
    // the BF16 stage may run as one persistent cooperative launch per component (k_stage.cu):
    // only when this context's fits do not share the GPU with other fits, and until such a
    // launch was refused for lack of resident CTAs
    bool persist_ok = true;
    std::string persist_note;  // why the persistent stage was not used, when it was refused
    // concurrent fits of ica_order_fit_batched: worker contexts with their own streams, and the
    // autotuned CTA share per (workers, shape) key
    std::vector<ica_ctx*> workers;
    std::vector<cudaStream_t> worker_streams;
    std::vector<std::pair<long long, int>> tuned;
};

// kinds of timed fused launches
// kinds of timed launches: the four fused kernels, then the remaining phases of a component
enum { K_ITER = 0, K_KURT = 1, K_REFINE = 2, K_REFKURT = 3, K_FINALIZE = 4, K_PRUNE = 5, K_BASIS = 6,
       K_REDUCE = 7, K_SELECT = 8, K_APPEND = 9, K_NKINDS = 10 };
static const char* kKindName[K_NKINDS] = {"iteration", "kurtosis", "refine", "refine_kurtosis", "finalize",
                                          "prune", "basis", "reduce", "select", "append"};

// Text of the last CUDA failure seen by this host thread (ica_last_error).
static thread_local std::string g_last_error;
static void note_cuda_error(cudaError_t e, const char* what, int line) {
    g_last_error = std::string(cudaGetErrorString(e)) + " in " + what + " (ica_api.cu:" + std::to_string(line) + ")";
}
#define CK(call)                                          \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) {                          \
            note_cuda_error(_e, #call, __LINE__);         \
            return ICA_ERR_CUDA;                          \
        }                                                 \
    } while (0)
// a launch of one of this library's kernels (counted)
#define KL(call)             \
    do {                     \
        CK(call);            \
        ++c->launches;       \
        ++c->launches_total; \
    } while (0)

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    int n_pad_max = 0, M_pad = 0, part_rows_max = 0;
    int64_t ldx = 0;
    size_t jscr;  // Jacobi scratch (mixed-precision solver above its shared-memory size)
    size_t W32;   // Algorithm 1: FP32 copy of the found components (N x n_pad_max)
    int64_t ld8 = 0;  // FP8: bytes per row of the E4M3 copy of X~
    size_t X8, fp8sc, rmax, zmax;  // FP8: E4M3 X~ (256 rows), its scales, row maxima, per-restart |z| maxima
    size_t status, counts, Xt32, Xt16, Z, B32, Bact, act0, act1, cand, flags, iters, traj, alpha, ups, excl, slots, pruned,
        part_acc, part_mom, G, jA, jV, lam, t1, t2, t3, t4, cov_part, comp_stats, comp_rows, total;
};

Layout make_layout(int N, int64_t T, int M, int precision) {
    Layout L;
    L.n_pad_max = round_up(N, 16);
    L.M_pad = round_up(M, kTcRows);
    L.ldx = round_up64(T, 8);
    L.part_rows_max = kMaxCTAs * kTcRows;
    if (L.part_rows_max < L.M_pad) L.part_rows_max = L.M_pad;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    const size_t nN = static_cast<size_t>(N) * N;
    L.status = take(16 * sizeof(int));
    L.counts = take(32 * sizeof(int));
    L.Xt32 = take(sizeof(float) * L.n_pad_max * static_cast<size_t>(L.ldx));
    const bool tc = precision == ICA_BF16 || precision == ICA_FP8;
    L.Xt16 = take(tc ? sizeof(uint16_t) * L.n_pad_max * static_cast<size_t>(L.ldx) : 0);
    const bool f8 = precision == ICA_FP8;
    L.ld8 = round_up64(T, 16);
    const int n8_max = (N + 31) / 32 * 32;
    L.X8 = take(f8 ? static_cast<size_t>(n8_max) * static_cast<size_t>(L.ld8) : 0);
    L.fp8sc = take(f8 ? sizeof(float) * (3 * 256 + 1) : 0);
    L.rmax = take(f8 ? sizeof(unsigned) * 256 : 0);
    L.zmax = take(f8 ? sizeof(float) * L.M_pad : 0);
    L.Z = take(precision == ICA_PLAIN_FP32 ? sizeof(float) * static_cast<size_t>(M) * L.ldx : 0);
    L.B32 = take(sizeof(float) * static_cast<size_t>(L.M_pad) * L.n_pad_max);
    L.Bact = take(precision == ICA_PLAIN_FP32 ? sizeof(float) * static_cast<size_t>(L.M_pad) * L.n_pad_max : 0);
    L.act0 = take(sizeof(int) * L.M_pad);
    L.act1 = take(sizeof(int) * L.M_pad);
    L.cand = take(sizeof(int) * 64);
    L.flags = take(sizeof(int) * L.M_pad);
    L.iters = take(sizeof(int) * L.M_pad);
    L.traj = take(sizeof(float) * L.M_pad * kTrajLen * 2);
    L.alpha = take(sizeof(double) * L.M_pad);
    L.ups = take(sizeof(double) * L.M_pad);
    L.excl = take(sizeof(int) * L.M_pad);
    L.slots = take(sizeof(int) * 64);
    L.pruned = take(sizeof(int) * L.M_pad);
    L.part_acc = take(sizeof(float) * static_cast<size_t>(L.part_rows_max) * L.n_pad_max);
    L.part_mom = take(sizeof(float) * static_cast<size_t>(L.part_rows_max) * 4);
    L.G = take(sizeof(double) * nN);
    L.jA = take(sizeof(double) * nN);
    L.jV = take(sizeof(double) * nN);
    L.lam = take(sizeof(double) * N);
    L.t1 = take(sizeof(double) * nN);
    L.t2 = take(sizeof(double) * nN);
    L.t3 = take(sizeof(double) * nN);
    L.t4 = take(sizeof(double) * nN);
    L.jscr = take(jacobi_scratch_bytes(N));
    L.W32 = take(sizeof(float) * static_cast<size_t>(N) * L.n_pad_max);
    L.cov_part = take(sizeof(double) * nN * covariance_splits(N, T));
    L.comp_stats = take(sizeof(double) * 4 * (N + 1));
    L.comp_rows = take(sizeof(long long) * 2 * (N + 1));  // per component: rows updated (stage, refine)
    L.total = off;
    return L;
}

template <typename P>
inline P* at(ica_ctx* c, size_t off) {
    return reinterpret_cast<P*>(c->ws + off);
}

int map_device_status(int st) {
    if (st & DEV_TIMEOUT) return ICA_ERR_TIMEOUT;
    if (st & DEV_ILLCOND) return ICA_ERR_ILLCOND;
    if (st & DEV_NONFINITE) return ICA_ERR_NONFINITE;
    if (st & DEV_ALLDEAD) return ICA_ERR_NONFINITE;
    return ICA_OK;
}

// Split of the sample range: about two waves of CTAs over the SMs, capped by kMaxCTAs.
void choose_splits(int64_t total_chunks, int tiles, int waves_ctas, int max_splits, int* splits, int* cps,
                   bool one_wave = false) {
    // one_wave: never more CTAs than the target (one CTA per SM): a partial second wave runs a
    // few CTAs alone for a whole CTA's time (measured on GB300, n = 128, M = 4096, T = 1e6:
    // 32 tiles x 5 splits = 160 CTAs 3.13 ms, 32 x 4 = 128 CTAs 1.91 ms)
    int s = one_wave && tiles <= waves_ctas ? waves_ctas / tiles : (waves_ctas + tiles - 1) / tiles;
    const int cap = kMaxCTAs / tiles > 0 ? kMaxCTAs / tiles : 1;
    if (s > cap) s = cap;
    if (max_splits > 0 && s > max_splits) s = max_splits;
    if (s < 1) s = 1;
    if (s > total_chunks) s = static_cast<int>(total_chunks);
    const int64_t c = (total_chunks + s - 1) / s;
    *cps = static_cast<int>(c);
    *splits = static_cast<int>((total_chunks + c - 1) / c);
}

int encode_xmap(ica_ctx* c, CUtensorMap* map, const uint16_t* Xt16, int n_pad, int64_t T, int64_t ld) {
    if (!c->encode) return ICA_ERR_UNSUPPORTED;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(T), static_cast<cuuint64_t>(n_pad)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
    cuuint32_t box[2] = {64u, static_cast<cuuint32_t>(n_pad)};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult r = c->encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(Xt16), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? ICA_OK : ICA_ERR_CUDA;
}

// E4M3 copy of X~ (n8 rows of ld bytes): boxes of 128 samples x n8 rows, 128-byte swizzle.
int encode_xmap8(ica_ctx* c, CUtensorMap* map, const uint8_t* X8, int n8, int64_t T, int64_t ld) {
    if (!c->encode) return ICA_ERR_UNSUPPORTED;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(T), static_cast<cuuint64_t>(n8)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld)};
    cuuint32_t box[2] = {128u, static_cast<cuuint32_t>(n8)};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult r = c->encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(X8), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? ICA_OK : ICA_ERR_CUDA;
}

int ensure_cublas(ica_ctx* c) {
    if (c->cublas) return ICA_OK;
    if (!c->cublas_lib) {
        c->cublas_lib = dlopen("libcublas.so.13", RTLD_NOW | RTLD_LOCAL);
        if (!c->cublas_lib) c->cublas_lib = dlopen("libcublas.so", RTLD_NOW | RTLD_LOCAL);
        if (!c->cublas_lib) return ICA_ERR_UNSUPPORTED;
    }
    auto create = reinterpret_cast<PFN_cublasCreate_t>(dlsym(c->cublas_lib, "cublasCreate_v2"));
    c->cublas_destroy = reinterpret_cast<PFN_cublasDestroy_t>(dlsym(c->cublas_lib, "cublasDestroy_v2"));
    c->cublas_set_stream = reinterpret_cast<PFN_cublasSetStream_t>(dlsym(c->cublas_lib, "cublasSetStream_v2"));
    c->sgemm = reinterpret_cast<PFN_cublasSgemm_t>(dlsym(c->cublas_lib, "cublasSgemm_v2"));
    if (!create || !c->cublas_destroy || !c->cublas_set_stream || !c->sgemm) return ICA_ERR_UNSUPPORTED;
    if (create(&c->cublas) != 0) {
        c->cublas = nullptr;
        return ICA_ERR_UNSUPPORTED;
    }
    return ICA_OK;
}

// One fused launch over the active rows -> split-T partial sums in the workspace.
struct StepShape {
    int splits = 1, cps = 1, part_rows = 0;
};

struct FusedArgs {
    int precision = ICA_BF16;
    bool moments_only = false;  // kurtosis pass: moments only, no update
    bool moments = true;        // update pass: also accumulate sum z^2, sum z^4
    const float* B32 = nullptr;
    int ldb = 0;
    const int* act = nullptr;        // active restart ids (NULL: rows 0..M_act-1)
    const int* count_dev = nullptr;  // device count of active rows (NULL: M_act is exact)
    int M_act = 0;                   // host upper bound of the active count (sizes the grid)
    int n_pad = 0;
    int64_t T = 0;
    const float* Xt32 = nullptr;
    const uint16_t* Xt16 = nullptr;
    int64_t ldx = 0;
    int max_splits = 0;
    int* shape_dev = nullptr;  // BF16 update: shape the launch on the device, write {splits, part_rows} here
    bool use_lo = true;        // BF16 update: the restart rows' low BF16 term enters the first product
    bool pdl = false;          // FP32 few-row update: programmatic dependent launch after the previous kernel
};

int run_fused(ica_ctx* c, const Layout& L, const FusedArgs& a, StepShape* shape) {
    cudaStream_t s = c->stream;
    float* pacc = at<float>(c, L.part_acc);
    float* pmom = at<float>(c, L.part_mom);
    int* status = at<int>(c, L.status);
    if (a.precision == ICA_BF16) {
        const int TC = tc_chunk(a.n_pad);
        const int64_t total = (a.T + TC - 1) / TC;
        const int tiles = (a.M_act + kTcRows - 1) / kTcRows;
        if (a.shape_dev && a.count_dev && !a.moments_only && a.max_splits == 0) {
            CUtensorMap map;
            int rc = encode_xmap(c, &map, a.Xt16, a.n_pad, a.T, a.ldx);
            if (rc) return rc;
            KL(launch_fused_tc_shaped(s, a.moments, map, a.B32, a.ldb, a.act, a.count_dev, a.M_act, a.n_pad, a.T,
                                      152 / c->cta_div, static_cast<int>(total), pacc, pmom, status, a.shape_dev,
                                      a.use_lo));
            shape->splits = -1;  // on the device (a.shape_dev)
            shape->cps = -1;
            shape->part_rows = -1;
            return ICA_OK;
        }
        choose_splits(total, tiles, 152 / c->cta_div, a.max_splits, &shape->splits, &shape->cps, true);  // one wave
        shape->part_rows = tiles * kTcRows;
        CUtensorMap map;
        int rc = encode_xmap(c, &map, a.Xt16, a.n_pad, a.T, a.ldx);
        if (rc) return rc;
        KL(launch_fused_tc(s, a.moments_only, a.moments, map, a.B32, a.ldb, a.act,
                           a.count_dev, a.M_act, a.n_pad, a.T, shape->splits, shape->cps, static_cast<int>(total), pacc,
                           pmom, shape->part_rows, status));
        return ICA_OK;
    }
    if (a.precision == ICA_FP32) {
        const int64_t total = (a.T + 63) / 64;
        if (a.M_act <= kFp32SmallRows) {  // a few candidates: bound by streaming X~
            const int64_t total_rows_chunks = (a.T + fp32_rows_chunk(a.n_pad) - 1) / fp32_rows_chunk(a.n_pad);
            choose_splits(total_rows_chunks, 1, 2 * 152 / c->cta_div, a.max_splits, &shape->splits, &shape->cps);
            shape->part_rows = fp32_rows_tile(a.M_act);
            KL(launch_fused_fp32_rows(s, a.moments_only, a.B32, a.ldb, a.act, a.count_dev, a.M_act, a.Xt32, a.ldx,
                                      a.n_pad, a.T, shape->splits, shape->cps, pacc, pmom, shape->part_rows, a.pdl));
            return ICA_OK;
        }
        const int tiles = (a.M_act + kFp32Rows - 1) / kFp32Rows;
        choose_splits(total, tiles, 4 * 152 / c->cta_div, a.max_splits, &shape->splits, &shape->cps);
        shape->part_rows = tiles * kFp32Rows;
        KL(launch_fused_fp32(s, a.moments_only, a.B32, a.ldb, a.act, a.count_dev, a.M_act, a.Xt32, a.ldx, a.n_pad,
                             a.T, shape->splits, shape->cps, pacc, pmom, shape->part_rows));
        return ICA_OK;
    }
    // plain FP32 matrix form: Z = B X~ in device memory, cube, second product (cuBLAS)
    int rc = ensure_cublas(c);
    if (rc) return rc;
    float* Bact = at<float>(c, L.Bact);
    float* Z = at<float>(c, L.Z);
    const int rows = a.M_act;
    KL(launch_gather_rows(s, a.B32, a.ldb, a.act, a.count_dev, rows, a.n_pad, Bact));
    if (c->cublas_set_stream(c->cublas, s) != 0) return ICA_ERR_CUDA;
    const float one = 1.f, zero = 0.f;
    if (c->sgemm(c->cublas, 0, 0, static_cast<int>(a.T), rows, a.n_pad, &one, a.Xt32, static_cast<int>(a.ldx), Bact,
                 a.n_pad, &zero, Z, static_cast<int>(a.ldx)) != 0)
        return ICA_ERR_CUDA;
    shape->splits = 1;
    shape->cps = 1;
    shape->part_rows = rows;
    if (a.moments_only) {
        KL(launch_row_moments(s, Z, rows, a.T, a.ldx, pmom));
        return ICA_OK;
    }
    KL(launch_cube_inplace(s, Z, rows, a.T, a.ldx));
    if (c->sgemm(c->cublas, 1, 0, a.n_pad, rows, static_cast<int>(a.T), &one, a.Xt32, static_cast<int>(a.ldx), Z,
                 static_cast<int>(a.ldx), &zero, pacc, a.n_pad) != 0)
        return ICA_ERR_CUDA;
    return ICA_OK;
}

// Host reads of the device active count after iteration t (1-based): every iteration at
// first, when most restarts leave, then every second, then every fourth. Between reads the
// launches are sized for the last count read, an upper bound (counts only fall).
bool sync_due(int t) { return t <= 4 || (t <= 12 && t % 2 == 0) || t % 4 == 0; }
// The BF16 stage shapes its launches on the device, so the host reads the count only to stop
// early when every restart converged.
bool sync_due_shaped(int t) { return t % 4 == 0; }

int check_ws(ica_ctx* c, const Layout& L) {
    if (!c->ws || c->ws_bytes < L.total) return ICA_ERR_WORKSPACE;
    return ICA_OK;
}

int read_status(ica_ctx* c, const Layout& L) {
    CK(cudaMemcpyAsync(c->host_i + 1, at<int>(c, L.status), sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return map_device_status(c->host_i[1]);
}

// Section 3.3: G = (F~F~^T)^(-1/2) F~ with F~ the first n = N - k rows of I - W^T W. With
// U = W[:, :n], F~F~^T = I_n - U^T U; its eigenproblem is solved on the smaller of the two
// Gram matrices:
//   k <= n: U U^T = Q diag(mu) Q^T (k x k) and (I - U^T U)^(-1/2) = I + U^T H U with
//           H = Q diag(f(mu)) Q^T, f(mu) = ((1 - mu)^(-1/2) - 1) / mu, so
//           G = F~ + U^T H U F~ = E_n + U^T (H (U~ - U U^T W) - W), U~ = [U 0];
//   k >  n: S = F~ F~^T = Q diag(l) Q^T (n x n, formed from the computed F~ so that G G^T = I
//           holds to rounding), G = Q diag(l^(-1/2)) Q^T F~.
// Smallest eigenvalue of F~F~^T (Eq. 7) accepted for the deflation basis. Keeping the first n
// rows of F makes F~F~^T = I - W_{:,:n}^T W_{:,:n} nearly singular when the found components
// nearly contain a unit vector of the first n coordinates; where the two subspaces have about equal
// dimension (i near N / 2) eigenvalues of 1e-11 occur in generic data. With FP64 eigenpairs
// (absolute error about 1e-16) an eigenvalue of 1e-14 still sets G's length along its eigenvector
// to within 1 % and its direction to within 1e-9, so only eigenvalues below that are an error.
constexpr double kBasisIllCond = 1e-14;

int deflation_basis_impl(ica_ctx* c, const Layout& L, const double* W, int k, int N, double* G) {
    cudaStream_t s = c->stream;
    const int n = N - k;
    double *A = at<double>(c, L.jA), *V = at<double>(c, L.jV), *lam = at<double>(c, L.lam);
    double *T1 = at<double>(c, L.t1), *T2 = at<double>(c, L.t2), *T3 = at<double>(c, L.t3), *T4 = at<double>(c, L.t4);
    int* status = at<int>(c, L.status);
    if (k == 0) {
        KL(launch_set_identity(s, G, N, N, N, 1.0));
        return ICA_OK;
    }
    if (k <= n) {
        KL(launch_gemm_f64(s, k, k, n, 1.0, W, N, 1, W, 1, N, 0.0, A, k));   // U U^T
        KL(launch_gemm_f64(s, k, k, n, 1.0, W, N, 1, W, 1, N, 0.0, T4, k));  // kept copy
        KL(launch_jacobi(s, A, V, lam, k, status, 60, c->ws + L.jscr));
        KL(launch_scale_cols_fn(s, V, lam, k, 1, T1, status, kBasisIllCond));  // Q f(mu)
        KL(launch_gemm_f64(s, k, k, k, 1.0, T1, k, 1, V, 1, k, 0.0, T2, k));  // H = Q f Q^T
        KL(launch_pad_cols(s, W, k, N, n, T3));                              // U~ = [U 0]
        KL(launch_gemm_f64(s, k, N, k, -1.0, T4, k, 1, W, N, 1, 1.0, T3, N));  // Y = U~ - (U U^T) W
        KL(launch_gemm_f64(s, k, N, k, 1.0, T2, k, 1, T3, N, 1, 0.0, T1, N));  // H Y
        KL(launch_axpby_f64(s, static_cast<int64_t>(k) * N, 1.0, T1, -1.0, W, T1));  // H Y - W
        KL(launch_set_identity(s, G, n, N, N, 1.0));                         // E_n
        KL(launch_gemm_f64(s, n, N, k, 1.0, W, 1, N, T1, N, 1, 1.0, G, N));  // + U^T (H Y - W)
        return ICA_OK;
    }
    KL(launch_set_identity(s, T3, n, N, N, 1.0));
    KL(launch_gemm_f64(s, n, N, k, -1.0, W, 1, N, W, N, 1, 1.0, T3, N));  // F~ = E_n - U^T W
    KL(launch_gemm_f64(s, n, n, N, 1.0, T3, N, 1, T3, 1, N, 0.0, A, n));  // S = F~ F~^T (Gram form)
    KL(launch_jacobi(s, A, V, lam, n, status, 60, c->ws + L.jscr));
    KL(launch_scale_cols_fn(s, V, lam, n, 0, T1, status, kBasisIllCond));
    KL(launch_gemm_f64(s, n, n, n, 1.0, T1, n, 1, V, 1, n, 0.0, T2, n));  // S^(-1/2)
    KL(launch_gemm_f64(s, n, N, n, 1.0, T2, n, 1, T3, N, 1, 0.0, G, N));  // G = S^(-1/2) F~
    return ICA_OK;
}

// Event pool for per-launch timing (profile option). Events are host-side driver objects.
int ev_take(ica_ctx* c, size_t* cursor) {
    if (*cursor >= c->ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        c->ev.push_back(e);
    }
    return static_cast<int>((*cursor)++);
}

// Accumulate the elapsed times of the recorded launches (after a stream synchronisation).
void harvest(ica_ctx* c) {
    for (const auto& r : c->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[r.e0], c->ev[r.e1]) == cudaSuccess) {
            c->kind_ms[r.kind] += ms;
            c->kind_flops[r.kind] += r.flops;
            c->kind_n[r.kind] += 1;
        }
    }
    c->recs.clear();
}

void json_kv(std::string& s, const char* k, double v, bool comma = true) {
    char buf[96];
    snprintf(buf, sizeof(buf), "\"%s\": %.10g%s", k, v, comma ? ", " : "");
    s += buf;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
extern "C" {

void ica_default_opts(ica_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = ICA_BF16;
    o->gauss_test = 0;
    o->refine_topk = 4;
    o->refine_iters = 10;
    o->stage_tol = 1e-4;
    o->refine_tol = 1e-6;
    o->fp32_tol_floor = 1e-6;
    o->B0 = nullptr;
    o->max_splits = 0;
    o->prune_params = nullptr;
    o->prune_tau = 0.05f;
    o->record_features = nullptr;
    o->record_labels = nullptr;
    o->stage_persistent = 1;
    o->prune_keep_frac = 0.05f;
    o->prune_cos = 0.99f;
    o->algorithm = 2;
    o->stage_lo_from = 5;
    o->prune_gauss = 1;
    o->stage_streamk = 1;
    o->fp8_iters = 3;
}

const char* ica_status_string(int st) {
    switch (st) {
        case ICA_OK: return "ok";
        case ICA_ERR_ARG: return "invalid argument";
        case ICA_ERR_CUDA: return "CUDA error";
        case ICA_ERR_NONFINITE: return "non-finite or vanishing restart update";
        case ICA_ERR_ILLCOND: return "ill-conditioned matrix (singular covariance or F~F~^T)";
        case ICA_ERR_TIMEOUT: return "bounded device wait timed out";
        case ICA_ERR_WORKSPACE: return "workspace missing or too small";
        case ICA_ERR_UNSUPPORTED: return "unsupported precision or feature";
        default: return "unknown status";
    }
}

int ica_create(ica_ctx** out, int device) {
    if (!out) return ICA_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return ICA_ERR_CUDA;
    ica_ctx* c = new ica_ctx();
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return ICA_ERR_CUDA;
    }
    if (cudaMallocHost(&c->host_i, 128 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->host_d, 1024 * sizeof(double)) != cudaSuccess) {
        delete c;
        return ICA_ERR_CUDA;
    }
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        c->encode = reinterpret_cast<PFN_encodeTiled_t>(fn);
    *out = c;
    return ICA_OK;
}

int ica_destroy(ica_ctx* c) {
    if (!c) return ICA_OK;
    for (ica_ctx* w : c->workers) ica_destroy(w);
    for (cudaStream_t st : c->worker_streams) cudaStreamDestroy(st);
    if (c->cublas && c->cublas_destroy) c->cublas_destroy(c->cublas);
    if (c->cublas_lib) dlclose(c->cublas_lib);
    if (c->host_i) cudaFreeHost(c->host_i);
    if (c->host_d) cudaFreeHost(c->host_d);
    delete c;
    return ICA_OK;
}

int ica_set_stream(ica_ctx* c, void* stream) {
    if (!c) return ICA_ERR_ARG;
    c->stream = static_cast<cudaStream_t>(stream);
    return ICA_OK;
}

size_t ica_workspace_bytes(int N, int64_t T, int M, const ica_opts* opts) {
    if (N < 1 || N > kMaxN || T < 1 || M < 1 || M > 65536) return 0;
    ica_opts d;
    ica_default_opts(&d);
    const ica_opts* o = opts ? opts : &d;
    return make_layout(N, T, M, o->precision).total;
}

int ica_set_workspace(ica_ctx* c, void* p, size_t bytes) {
    if (!c) return ICA_ERR_ARG;
    if (p && (reinterpret_cast<uintptr_t>(p) % kAlign) != 0) return ICA_ERR_ARG;
    c->ws = static_cast<uint8_t*>(p);
    c->ws_bytes = p ? bytes : 0;
    return ICA_OK;
}

int ica_whiten(ica_ctx* c, const float* X, int N, int64_t T, float* Xw, double* V, double* mean) {
    if (!c || !X || !Xw || !V || !mean || N < 1 || N > kMaxN || T < 2 * static_cast<int64_t>(N)) return ICA_ERR_ARG;
    if (reinterpret_cast<const void*>(X) == reinterpret_cast<const void*>(Xw)) return ICA_ERR_ARG;
    const Layout L = make_layout(N, T, 1, ICA_FP32);
    int rc = check_ws(c, L);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    int* status = at<int>(c, L.status);
    CK(cudaMemsetAsync(status, 0, sizeof(int), s));
    double *A = at<double>(c, L.jA), *E = at<double>(c, L.jV), *lam = at<double>(c, L.lam);
    double *T1 = at<double>(c, L.t1), *bias = at<double>(c, L.t2);
    const int splits = covariance_splits(N, T);
    KL(launch_row_mean(s, X, N, T, T, mean, status));
    KL(launch_covariance(s, X, mean, N, T, T, at<double>(c, L.cov_part), splits, A));
    ++c->launches;  // partial + reduce
    ++c->launches_total;
    KL(launch_jacobi(s, A, E, lam, N, status, 60, c->ws + L.jscr));
    KL(launch_scale_cols_fn(s, E, lam, N, 0, T1, status, 1e-12));
    KL(launch_gemm_f64(s, N, N, N, 1.0, T1, N, 1, E, 1, N, 0.0, V, N));     // V = E diag(l^-1/2) E^T
    KL(launch_gemm_f64(s, N, 1, N, 1.0, V, N, 1, mean, 1, 1, 0.0, bias, 1));  // V mean
    KL(launch_rows_gemm(s, V, N, N, N, X, T, T, bias, Xw, T, nullptr, 0));
    CK(cudaMemcpyAsync(c->host_i + 1, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // NaN or Inf in X also breaks the eigendecomposition: report the cause, not the symptom
    if (c->host_i[1] & DEV_NONFINITE) return ICA_ERR_NONFINITE;
    return map_device_status(c->host_i[1]);
}

int ica_init_restarts(ica_ctx* c, uint64_t seed, int component, int M, int n, float* B, int ldb) {
    if (!c || !B || M < 1 || n < 1 || n > kMaxN || ldb < n || component < 0) return ICA_ERR_ARG;
    CK(cudaSetDevice(c->device));
    KL(launch_init_restarts(c->stream, seed, component, M, n, ldb, nullptr, 0, B));
    return ICA_OK;
}

int ica_deflation_basis(ica_ctx* c, const double* W, int k, int N, double* G) {
    if (!c || !G || N < 1 || N > kMaxN || k < 0 || k >= N || (k > 0 && !W)) return ICA_ERR_ARG;
    const Layout L = make_layout(N, 8, 1, ICA_FP32);
    int rc = check_ws(c, L);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    CK(cudaMemsetAsync(at<int>(c, L.status), 0, sizeof(int), c->stream));
    rc = deflation_basis_impl(c, L, W, k, N, G);
    if (rc) return rc;
    return read_status(c, L);
}

int ica_reduce(ica_ctx* c, const double* G, int n, int N, const float* Xw, int64_t T, float* Xt32, int64_t ldx32,
               uint16_t* Xt16, int64_t ldx16) {
    if (!c || !G || !Xw || n < 1 || n > N || N > kMaxN || T < 1) return ICA_ERR_ARG;
    if ((Xt32 && (ldx32 < T || ldx32 % 8)) || (Xt16 && (ldx16 < T || ldx16 % 8))) return ICA_ERR_ARG;
    CK(cudaSetDevice(c->device));
    KL(launch_rows_gemm(c->stream, G, n, round_up(n, 16), N, Xw, T, T, nullptr, Xt32, ldx32, Xt16, ldx16));
    return ICA_OK;
}

int ica_quantize_e4m3(ica_ctx* c, const float* Xt32, int n, int64_t T, int64_t ldx32, uint8_t* X8, int64_t ld8,
                      float* scales) {
    if (!c || !Xt32 || !X8 || !scales || n < 1 || n > kMaxN || T < 1 || ldx32 < T || ldx32 % 8 || ld8 < T ||
        ld8 % 16)
        return ICA_ERR_ARG;
    const Layout L = make_layout(n, T, 1, ICA_FP8);
    int rc = check_ws(c, L);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    int extra = 0;
    CK(launch_fp8_copy(c->stream, Xt32, ldx32, T, n, (n + 31) / 32 * 32, at<unsigned>(c, L.rmax), scales, X8, ld8,
                       &extra));
    c->launches += extra;
    c->launches_total += extra;
    return ICA_OK;
}

int ica_fp_step(ica_ctx* c, int precision, const float* B, int M, int n, const void* Xt, int64_t T, int64_t ldx,
                float* Bnew, float* moments) {
    if (!c || !B || !Xt || !Bnew || M < 1 || M > 65536 || n < 1 || n > kMaxN || T < 1 || ldx < T || ldx % 8)
        return ICA_ERR_ARG;
    if (precision != ICA_FP32 && precision != ICA_BF16) return ICA_ERR_UNSUPPORTED;
    const Layout L = make_layout(n, T, M, precision);
    int rc = check_ws(c, L);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    const int n_pad = round_up(n, 16);
    CK(cudaMemsetAsync(at<int>(c, L.status), 0, sizeof(int), c->stream));
    StepShape sh;
    FusedArgs fa;
    fa.precision = precision;
    fa.B32 = B;
    fa.ldb = n_pad;
    fa.M_act = M;
    fa.n_pad = n_pad;
    fa.T = T;
    fa.Xt32 = static_cast<const float*>(Xt);
    fa.Xt16 = static_cast<const uint16_t*>(Xt);
    fa.ldx = ldx;
    rc = run_fused(c, L, fa, &sh);
    if (rc) return rc;
    KL(launch_combine(c->stream, at<float>(c, L.part_acc), at<float>(c, L.part_mom), sh.splits, sh.part_rows, n_pad,
                      M, B, 1.0 / static_cast<double>(T), Bnew, moments));
    return read_status(c, L);
}

int ica_kurtosis(ica_ctx* c, int precision, const float* B, int M, int n, const void* Xt, int64_t T, int64_t ldx,
                 double* alpha, double* ups) {
    if (!c || !B || !Xt || !alpha || !ups || M < 1 || M > 65536 || n < 1 || n > kMaxN || T < 1 || ldx < T ||
        ldx % 8)
        return ICA_ERR_ARG;
    if (precision != ICA_FP32 && precision != ICA_BF16) return ICA_ERR_UNSUPPORTED;
    const Layout L = make_layout(n, T, M, precision);
    int rc = check_ws(c, L);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    const int n_pad = round_up(n, 16);
    CK(cudaMemsetAsync(at<int>(c, L.status), 0, sizeof(int), c->stream));
    StepShape sh;
    FusedArgs fa;
    fa.precision = precision;
    fa.moments_only = true;
    fa.B32 = B;
    fa.ldb = n_pad;
    fa.M_act = M;
    fa.n_pad = n_pad;
    fa.T = T;
    fa.Xt32 = static_cast<const float*>(Xt);
    fa.Xt16 = static_cast<const uint16_t*>(Xt);
    fa.ldx = ldx;
    rc = run_fused(c, L, fa, &sh);
    if (rc) return rc;
    KL(launch_kurt_finalize(c->stream, at<float>(c, L.part_mom), sh.splits, sh.part_rows, nullptr, nullptr, M,
                            1.0 / static_cast<double>(T), alpha, ups));
    return read_status(c, L);
}

int ica_order_fit(ica_ctx* c, const float* Xw, int N, int64_t T, int M, int n_components, int iters, double tol,
                  uint64_t seed, const ica_opts* opts, double* W_out, double* kurt_out, int* n_found) {
    if (!c || !Xw || !W_out || !kurt_out || !n_found) return ICA_ERR_ARG;
    *n_found = 0;
    if (N < 1 || N > kMaxN || T < 2 * static_cast<int64_t>(N) || M < 1 || M > 65536 || n_components < 1 ||
        n_components > N || iters < 1 || !(tol > 0.0))
        return ICA_ERR_ARG;
    ica_opts d;
    ica_default_opts(&d);
    const ica_opts o = opts ? *opts : d;
    if (o.precision != ICA_FP32 && o.precision != ICA_BF16 && o.precision != ICA_FP8 && o.precision != ICA_PLAIN_FP32)
        return ICA_ERR_UNSUPPORTED;
    const bool tcp = o.precision == ICA_BF16 || o.precision == ICA_FP8;  // tensor-core stage + FP32 refinement
    if (tcp && (o.refine_topk < 1 || o.refine_topk > 32 || o.refine_iters < 1)) return ICA_ERR_ARG;
    if (o.wait_ns < 0 || (o.record_cands && !tcp) || o.fp8_iters < 0) return ICA_ERR_ARG;
    if (o.algorithm != 1 && o.algorithm != 2) return ICA_ERR_ARG;
    if (o.stage_lo_from < 0) return ICA_ERR_ARG;
    const bool alg1 = o.algorithm == 1;
    if (!(o.prune_keep_frac >= 0.f && o.prune_keep_frac <= 1.f) || !(o.prune_cos >= 0.f && o.prune_cos <= 1.f))
        return ICA_ERR_ARG;
    const Layout L = make_layout(N, T, M, o.precision);
    int rc = check_ws(c, L);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    const bool bf16 = tcp;  // the BF16 stage (and FP8 iterations inside it) + FP32 refinement
    // FP8: iterations 1..fp8_iters of each component's stage take E4M3 operands; iteration 0 (BF16)
    // records each restart's largest |z| for the scale of the first FP8 iteration's P. Needs the
    // persistent stage (the per-launch path runs those iterations in BF16).
    const int fp8_until = o.precision == ICA_FP8 && o.fp8_iters > 0 ? 1 + o.fp8_iters : 0;
    uint8_t* X8 = at<uint8_t>(c, L.X8);
    float* fp8sc = at<float>(c, L.fp8sc);
    float* zmax = at<float>(c, L.zmax);
    long long fp8_launches = 0;
    const double inv_T = 1.0 / static_cast<double>(T);
    int* status = at<int>(c, L.status);
    int* counts = at<int>(c, L.counts);  // [0], [1]: active counts (double-buffered); [2]: candidates
    unsigned int* done_ctr = reinterpret_cast<unsigned int*>(counts + 8);  // finalize's block counter
    unsigned int* stage_bar = reinterpret_cast<unsigned int*>(counts + 16);  // persistent stage's grid barrier
    int* stage_ctl = counts + 20;  // persistent stage's {iteration reached, active count, list index}
    float* B32 = at<float>(c, L.B32);
    float* Xt32 = at<float>(c, L.Xt32);
    uint16_t* Xt16 = at<uint16_t>(c, L.Xt16);
    int* act[2] = {at<int>(c, L.act0), at<int>(c, L.act1)};
    int* flags = at<int>(c, L.flags);
    int* itc = at<int>(c, L.iters);
    float* traj = at<float>(c, L.traj);
    double* alpha = at<double>(c, L.alpha);
    double* ups = at<double>(c, L.ups);
    int* excl = at<int>(c, L.excl);
    int* cand = at<int>(c, L.cand);
    int* cand_list = at<int>(c, L.slots) + 32;
    int* slots = at<int>(c, L.slots);
    double* G = at<double>(c, L.G);
    float* W32 = at<float>(c, L.W32);
    double* cstats = at<double>(c, L.comp_stats);
    long long* crows = at<long long>(c, L.comp_rows);
    const int64_t ldx = L.ldx;
    const double tol_fp32 = tol > o.fp32_tol_floor ? tol : o.fp32_tol_floor;
    const double tol_iter = bf16 ? (o.stage_tol > tol ? o.stage_tol : tol) : tol_fp32;
    const double tol_ref = o.refine_tol > o.fp32_tol_floor ? o.refine_tol : o.fp32_tol_floor;
    const int refine_iters = o.refine_iters < iters ? o.refine_iters : iters;

    CK(cudaMemsetAsync(status, 0, sizeof(int), s));
    CK(cudaMemsetAsync(done_ctr, 0, sizeof(unsigned int), s));
    CK(cudaMemsetAsync(crows, 0, sizeof(long long) * 2 * (N + 1), s));
    c->launches = 0;
    for (int k = 0; k < K_NKINDS; ++k) {
        c->kind_ms[k] = 0.0;
        c->kind_flops[k] = 0.0;
        c->kind_n[k] = 0;
    }
    c->recs.clear();
    size_t ev_cursor = 0;
    // one fused launch, bracketed by CUDA events on the context stream when profiling; the
    // FLOP count uses the host's active count of the last read (an upper bound between reads)
    auto timed = [&](int kind, double flops, auto&& fn) -> int {
        if (!o.profile) return fn();
        const int e0 = ev_take(c, &ev_cursor), e1 = ev_take(c, &ev_cursor);
        if (e0 < 0 || e1 < 0) return ICA_ERR_CUDA;
        CK(cudaEventRecord(c->ev[e0], s));
        const int r = fn();
        CK(cudaEventRecord(c->ev[e1], s));
        c->recs.push_back({kind, flops, e0, e1});
        return r;
    };
    // read the device count of the active rows (and the status word) back to the host
    auto read_count = [&](const int* count_dev, int* out) -> int {
        CK(cudaMemcpyAsync(c->host_i, count_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(c->host_i + 1, status, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const int r = map_device_status(c->host_i[1]);
        if (r) return r;
        *out = c->host_i[0];
        return ICA_OK;
    };
    struct EventGuard {  // destroys the fit's two events on every return path
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~EventGuard() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } fit_ev;
    CK(cudaEventCreate(&fit_ev.e[0]));
    CK(cudaEventCreate(&fit_ev.e[1]));
    cudaEvent_t fit_begin = fit_ev.e[0], fit_end = fit_ev.e[1];
    CK(cudaEventRecord(fit_begin, s));
    const double dT = static_cast<double>(T);
    std::vector<int> comp_iters, comp_refine, comp_pruned, comp_fallback;
    std::vector<double> comp_stage_ms;  // per component: stage (update) time, when profiling
    std::vector<int> comp_kurt_rows;    // per component: rows of the kurtosis pass
    const bool prune_opt = o.prune_params != nullptr && o.precision != ICA_PLAIN_FP32;
    int* pruned = at<int>(c, L.pruned);
    float* uref = reinterpret_cast<float*>(counts + 12);  // pruner feature reference (one float)
    std::vector<std::vector<int>> comp_hist;
    long long persist_launches = 0;  // persistent BF16 stage launches of this fit
    int found = 0;
    for (int i = 0; i < n_components; ++i) {
        // Algorithm 2: reduced dimension n = N - i. Algorithm 1: every iteration on the full
        // whitened data (n = N, G = I, X~ = Xw, formed once), the found components projected out
        // of every update (Wp, the FP32 copy of W).
        const int n = alg1 ? N : N - i;
        const int n_pad = round_up(n, 16);
        const float* Wp = alg1 && i > 0 ? W32 : nullptr;
        if (!alg1 || i == 0) {
            // reduction basis and X~ = G Xw (Section 3.3)
            rc = timed(K_BASIS, 0.0, [&] { return deflation_basis_impl(c, L, W_out, i, N, G); });
            if (rc) return rc;
            rc = timed(K_REDUCE, 0.0, [&] {
                KL(launch_rows_gemm(s, G, n, n_pad, N, Xw, T, T, nullptr, Xt32, ldx, bf16 ? Xt16 : nullptr, ldx));
                if (fp8_until > 1) {  // E4M3 copy of X~ with per-row power-of-two scales
                    int extra = 0;
                    CK(launch_fp8_copy(s, Xt32, ldx, T, n, (n + 31) / 32 * 32, at<unsigned>(c, L.rmax), fp8sc, X8,
                                       L.ld8, &extra));
                    c->launches += extra;
                    c->launches_total += extra;
                }
                return ICA_OK;
            });
            if (rc) return rc;
        }
        // Attempt 0 may run the learned pruner after kTrajLen iterations; when the pruned restarts
        // look at least as good as the kept ones (prune_check), the component is fitted again
        // without pruning from the same initial restarts (attempt 1).
        int t = 0, rt = 0, n_pruned = 0, fell_back = 0;
        int kurt_rows = M;  // restarts whose kurtosis the component computed (all, or those the pruner kept)
        long long stage_rows_seen = 0;  // last value read of this component's stage row counter
        long long refine_rows_seen = 0;  // the same for its refinement row counter
        std::vector<int> hist;
        bool pruned_now = false, dropped_all = false;
        FusedArgs fa;
        for (int attempt = 0;; ++attempt) {
            const bool prune_this = prune_opt && attempt == 0;
            pruned_now = false;
            dropped_all = false;
            hist.clear();
            if (prune_opt) CK(cudaMemsetAsync(pruned, 0, sizeof(int) * M, s));
            // initial restarts
            KL(launch_init_restarts(s, seed, i, M, n, n_pad, o.B0 ? o.B0 + static_cast<int64_t>(i) * M * N : nullptr, N,
                                    B32));
            if (Wp) KL(launch_project_rows(s, B32, n_pad, M, n, Wp, i, n_pad));
            CK(cudaMemsetAsync(itc, 0, sizeof(int) * M, s));
            CK(cudaMemsetAsync(traj, 0, sizeof(float) * M * kTrajLen * 2, s));
            KL(launch_iota(s, act[0], M, counts + 0));
            fa = FusedArgs();
            fa.precision = bf16 ? ICA_BF16 : o.precision;
            fa.B32 = B32;
            fa.ldb = n_pad;
            fa.n_pad = n_pad;
            fa.T = T;
            fa.Xt32 = Xt32;
            fa.Xt16 = Xt16;
            fa.ldx = ldx;
            fa.max_splits = o.max_splits;
            // fixed-point iterations with removal of converged rows (Algorithm 2, Section 3.2)
            int cur = 0, M_host = M;
            t = 0;
            fa.shape_dev = bf16 ? counts + 14 : nullptr;  // {splits, part_rows} of each BF16 update
            // The BF16 stage runs as one persistent cooperative launch per segment of iterations
            // (k_stage.cu; same arithmetic as the per-launch path below) when the fit owns the GPU.
            bool persist = bf16 && o.stage_persistent && o.max_splits == 0 && c->persist_ok && c->cta_div == 1 &&
                           M <= 152 * kTcRows;
            while (t < iters && M_host > 0) {
                if (persist) {
                    // one launch per segment of iterations: [0, 1) BF16 and [1, fp8_until) FP8 in the
                    // FP8 form, [.., kTrajLen) up to the pruner, the rest
                    int t_end = (prune_this && t < kTrajLen) ? std::min(iters, kTrajLen) : iters;
                    const bool f8_now = fp8_until > 1 && t >= 1 && t < fp8_until;
                    if (fp8_until > 1) t_end = std::min(t_end, t < 1 ? 1 : (t < fp8_until ? fp8_until : t_end));
                    CUtensorMap map;
                    rc = f8_now ? encode_xmap8(c, &map, X8, (n + 31) / 32 * 32, T, L.ld8)
                                : encode_xmap(c, &map, Xt16, n_pad, T, ldx);
                    if (rc) return rc;
                    StageLaunch sl{};
                    sl.B32 = B32;
                    sl.ldb = n_pad;
                    sl.act0 = act[0];
                    sl.act1 = act[1];
                    sl.count0 = counts + 0;
                    sl.count1 = counts + 1;
                    sl.cur0 = cur;
                    sl.n_pad = n_pad;
                    sl.n = n;
                    sl.T = T;
                    sl.ctas = 152;
                    sl.part_acc = at<float>(c, L.part_acc);
                    sl.part_mom = at<float>(c, L.part_mom);
                    sl.flags = flags;
                    sl.iters = itc;
                    sl.traj = traj;
                    sl.status = status;
                    sl.rows_accum = crows + 2 * i;
                    sl.bar_ctr = stage_bar;
                    sl.ctl = stage_ctl;
                    sl.t_begin = t;
                    sl.t_end = t_end;
                    sl.inv_T = inv_T;
                    sl.tol = tol_iter;
                    sl.wait_ns = static_cast<uint64_t>(o.wait_ns);
                    sl.stall = o.stall_test != 0;
                    sl.Wp = Wp;
                    sl.nw = i;
                    sl.ldw = n_pad;
                    sl.lo_from = o.stage_lo_from;
                    sl.streamk = o.stage_streamk;
                    sl.fp8 = f8_now;
                    sl.zmax = fp8_until > 1 ? zmax : nullptr;
                    sl.track_until = fp8_until;
                    sl.fp8sc = fp8sc;
                    if (f8_now) ++fp8_launches;
                    CK(cudaMemsetAsync(stage_bar, 0, sizeof(unsigned int), s));
                    cudaError_t le = cudaSuccess;
                    int resident = 0;
                    const size_t rec0 = c->recs.size();
                    rc = timed(K_ITER, 0.0, [&] {
                        le = launch_stage_tc(s, map, sl, &resident);
                        return ICA_OK;
                    });
                    if (rc) return rc;
                    if (le == cudaErrorCooperativeLaunchTooLarge) {  // not all CTAs can be resident
                        cudaGetLastError();
                        c->persist_ok = false;
                        c->persist_note = "cooperative launch too large: " + std::to_string(resident) +
                                          " resident CTAs at n_pad " + std::to_string(n_pad);
                        persist = false;
                        if (c->recs.size() > rec0) c->recs.pop_back();
                        continue;
                    }
                    if (le != cudaSuccess) {
                        note_cuda_error(le, "launch_stage_tc", __LINE__);
                        return ICA_ERR_CUDA;
                    }
                    ++c->launches;
                    ++c->launches_total;
                    ++persist_launches;
                    long long* rows_h = reinterpret_cast<long long*>(c->host_i + 100);
                    CK(cudaMemcpyAsync(c->host_i + 96, stage_ctl, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
                    CK(cudaMemcpyAsync(c->host_i + 1, status, sizeof(int), cudaMemcpyDeviceToHost, s));
                    CK(cudaMemcpyAsync(rows_h, crows + 2 * i, sizeof(long long), cudaMemcpyDeviceToHost, s));
                    const long long rows_before = stage_rows_seen;
                    CK(cudaStreamSynchronize(s));
                    rc = map_device_status(c->host_i[1]);
                    if (rc) return rc;
                    t = c->host_i[96];
                    M_host = c->host_i[97];
                    cur = c->host_i[98];
                    stage_rows_seen = *rows_h;
                    if (c->recs.size() > rec0)  // exact FLOPs of the segment: rows updated x 4 n T
                        c->recs.back().flops = 4.0 * n * static_cast<double>(*rows_h - rows_before) * dT;
                    hist.push_back(M_host);
                }
                if (!persist) {
                    StepShape sh;
                    fa.act = act[cur];
                    fa.count_dev = counts + cur;
                    fa.M_act = M_host;
                    fa.moments_only = false;
                    fa.moments = t < kTrajLen;
                    fa.use_lo = t >= o.stage_lo_from;
                    rc = timed(K_ITER, 4.0 * n * M_host * dT, [&] { return run_fused(c, L, fa, &sh); });
                    if (rc) return rc;
                    rc = timed(K_FINALIZE, 0.0, [&] {
                        KL(launch_finalize(s, at<float>(c, L.part_acc), at<float>(c, L.part_mom), sh.splits, sh.part_rows,
                                           n_pad, n, act[cur], counts + cur, M_host, B32, n_pad, inv_T, tol_iter, flags, itc,
                                           o.precision == ICA_PLAIN_FP32 ? nullptr : traj, t, status, act[cur ^ 1],
                                           counts + (cur ^ 1), crows + 2 * i, done_ctr, fa.shape_dev,
                                           fa.shape_dev != nullptr,
                                           // the persistent stage's summation order when this
                                           // context may run it (identical results either way),
                                           // else four virtual warps per row
                                           fa.shape_dev && c->cta_div == 1 ? 152 : 0, Wp, i, n_pad));
                        return ICA_OK;
                    });
                    if (rc) return rc;
                    cur ^= 1;
                    ++t;
                    if (fa.shape_dev ? sync_due_shaped(t) : sync_due(t)) {
                        rc = read_count(counts + cur, &M_host);
                        if (rc) return rc;
                        hist.push_back(M_host);
                    }
                }
                if (prune_this && t == kTrajLen && t < iters) {
                    // learned pruner on the first kTrajLen iterations' trajectories
                    int before = M_host;
                    rc = timed(K_PRUNE, 0.0, [&] {
                        // Eq. 3 for component i + 1: Upsilon below 2 (N - i + 1)(N - i) / T
                        const float gthr = o.prune_gauss
                                               ? static_cast<float>(2.0 * (N - i + 1) * (N - i) / static_cast<double>(T))
                                               : 0.f;
                        KL(launch_prune(s, o.prune_params, traj, act[cur], counts + cur, M_host, N - i,
                                        std::log(static_cast<double>(T)), o.prune_tau, gthr, uref, flags, pruned,
                                        o.prune_keep_frac > 0.f ? (bf16 ? o.refine_topk : 1) : 0,
                                        o.prune_keep_frac, B32, n_pad, n, o.prune_cos, excl));
                        KL(launch_compact_keep(s, flags, act[cur], counts + cur, M_host, act[cur ^ 1], counts + (cur ^ 1)));
                        return ICA_OK;
                    });
                    if (rc) return rc;
                    cur ^= 1;
                    rc = read_count(counts + (cur ^ 1), &before);  // exact count before pruning
                    if (rc) return rc;
                    rc = read_count(counts + cur, &M_host);
                    if (rc) return rc;
                    n_pruned = before - M_host;
                    hist.push_back(M_host);
                    pruned_now = true;
                    dropped_all = before > 0 && M_host == 0;
                }
            }
            fa.shape_dev = nullptr;
            fa.use_lo = true;
            // kurtosis of every candidate: converged rows plus rows still running after `iters`
            // (after pruning: the restarts that stayed; the pruned ones leave the pick)
            {
                StepShape sh;
                int* kept_list = pruned_now ? act[cur ^ 1] : nullptr;
                int kept = M;
                if (pruned_now) {  // the grid is sized for the exact count of restarts that stayed
                    KL(launch_compact_keep(s, pruned, nullptr, nullptr, M, kept_list, counts + 6, true));
                    rc = read_count(counts + 6, &kept);
                    if (rc) return rc;
                }
                kurt_rows = kept;
                fa.act = kept_list;
                fa.count_dev = pruned_now ? counts + 6 : nullptr;
                fa.M_act = kept > 0 ? kept : 1;
                fa.moments_only = true;
                if (kept > 0) {
                    rc = timed(K_KURT, 2.0 * n * kept * dT, [&] { return run_fused(c, L, fa, &sh); });
                    if (rc) return rc;
                    KL(launch_kurt_finalize(s, at<float>(c, L.part_mom), sh.splits, sh.part_rows, kept_list,
                                            fa.count_dev, kept, inv_T, alpha, ups));
                }
            }
            if (!pruned_now) break;
            int fb = 0;
            KL(launch_prune_check(s, ups, pruned, traj, M, counts + 4));
            rc = read_count(counts + 4, &fb);
            if (rc) return rc;
            if (!fb && !dropped_all) break;
            fell_back = 1;  // the pruned restarts may hold the optimum: refit without pruning
        }
        const int* excl0 = pruned_now ? pruned : nullptr;  // restarts dropped by the pruner
        if (!bf16) {
            KL(launch_argmax(s, ups, excl0, nullptr, nullptr, M, slots));
        } else {
            // distinct top-k candidates, FP32 refinement, FP32 kurtosis, argmax among them
            const int k = o.refine_topk;
            rc = timed(K_SELECT, 0.0, [&] {
                KL(launch_select_clear(s, excl, excl0, M, cand, k));
                for (int j = 0; j < k; ++j) {
                    KL(launch_argmax(s, ups, excl, nullptr, nullptr, M, cand + j));
                    KL(launch_exclude(s, B32, n_pad, n, M, cand + j, excl, 1.0 - 1e-3));
                }
                KL(launch_compact_cand(s, cand, k, act[0], cand_list, counts + 2));
                return ICA_OK;
            });
            if (rc) return rc;
            CK(cudaMemcpyAsync(counts + 0, counts + 2, sizeof(int), cudaMemcpyDeviceToDevice, s));
            int rcur = 0, R_host = k;
            fa.precision = ICA_FP32;
            // persistent refinement (one cooperative launch for all its iterations; same
            // arithmetic as the per-launch loop below) when the fit has the GPU to itself
            bool rpersist = o.stage_persistent && c->persist_ok && c->cta_div == 1 && o.max_splits == 0 && k <= 4;
            while (rpersist && rt < refine_iters && R_host > 0) {
                const int64_t rchunks = (T + fp32_rows_chunk(n_pad) - 1) / fp32_rows_chunk(n_pad);
                StepShape rsh;
                choose_splits(rchunks, 1, 2 * 152, 0, &rsh.splits, &rsh.cps);
                RefineLaunch rl{};
                rl.B32 = B32;
                rl.ldb = n_pad;
                rl.act0 = act[0];
                rl.act1 = act[1];
                rl.count0 = counts + 0;
                rl.count1 = counts + 1;
                rl.cur0 = rcur;
                rl.Xt = Xt32;
                rl.ldx = ldx;
                rl.n_pad = n_pad;
                rl.n = n;
                rl.T = T;
                rl.splits = rsh.splits;
                rl.cps = rsh.cps;
                rl.rows_max = R_host;
                rl.part_acc = at<float>(c, L.part_acc);
                rl.part_mom = at<float>(c, L.part_mom);
                rl.flags = flags;
                rl.iters = itc;
                rl.status = status;
                rl.rows_accum = crows + 2 * i + 1;
                rl.bar_ctr = stage_bar;
                rl.ctl = stage_ctl;
                rl.t_begin = rt;
                rl.t_end = refine_iters;
                rl.inv_T = static_cast<float>(inv_T);
                rl.tol = static_cast<float>(tol_ref);
                rl.Wp = Wp;
                rl.nw = i;
                rl.ldw = n_pad;
                rl.wait_ns = static_cast<uint64_t>(o.wait_ns);
                CK(cudaMemsetAsync(stage_bar, 0, sizeof(unsigned int), s));
                cudaError_t le = cudaSuccess;
                int resident = 0;
                const size_t rec0 = c->recs.size();
                rc = timed(K_REFINE, 0.0, [&] {
                    le = launch_refine_fp32(s, rl, &resident);
                    return ICA_OK;
                });
                if (rc) return rc;
                if (le == cudaErrorCooperativeLaunchTooLarge) {  // not all CTAs can be resident
                    cudaGetLastError();
                    c->persist_ok = false;
                    c->persist_note = "refinement: cooperative launch too large: " + std::to_string(resident) +
                                      " resident CTAs";
                    if (c->recs.size() > rec0) c->recs.pop_back();
                    rpersist = false;
                    break;
                }
                if (le != cudaSuccess) {
                    note_cuda_error(le, "launch_refine_fp32", __LINE__);
                    return ICA_ERR_CUDA;
                }
                ++c->launches;
                ++c->launches_total;
                ++persist_launches;
                long long* rows_h = reinterpret_cast<long long*>(c->host_i + 100);
                CK(cudaMemcpyAsync(c->host_i + 96, stage_ctl, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
                CK(cudaMemcpyAsync(c->host_i + 1, status, sizeof(int), cudaMemcpyDeviceToHost, s));
                CK(cudaMemcpyAsync(rows_h, crows + 2 * i + 1, sizeof(long long), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                rc = map_device_status(c->host_i[1]);
                if (rc) return rc;
                if (c->recs.size() > rec0)  // exact FLOPs: rows updated x 4 n T
                    c->recs.back().flops = 4.0 * n * static_cast<double>(*rows_h - refine_rows_seen) * dT;
                refine_rows_seen = *rows_h;
                rt = c->host_i[96];
                R_host = c->host_i[97];
                rcur = c->host_i[98];
            }
            while (rt < refine_iters && R_host > 0) {
                StepShape sh;
                fa.act = act[rcur];
                fa.count_dev = counts + rcur;
                fa.M_act = R_host;
                fa.moments_only = false;
                fa.moments = false;
                fa.pdl = rt > 0;  // after the previous iteration's finalize (kernel to kernel)
                rc = timed(K_REFINE, 4.0 * n * R_host * dT, [&] { return run_fused(c, L, fa, &sh); });
                fa.pdl = false;
                if (rc) return rc;
                rc = timed(K_FINALIZE, 0.0, [&] {
                    KL(launch_finalize(s, at<float>(c, L.part_acc), at<float>(c, L.part_mom), sh.splits, sh.part_rows,
                                       n_pad, n, act[rcur], counts + rcur, R_host, B32, n_pad, inv_T, tol_ref, flags,
                                       itc, nullptr, kTrajLen, status, act[rcur ^ 1], counts + (rcur ^ 1),
                                       crows + 2 * i + 1, done_ctr, nullptr, true, 0, Wp, i, n_pad));
                    return ICA_OK;
                });
                if (rc) return rc;
                rcur ^= 1;
                ++rt;
                // launches size for the host bound and read the exact count on the device: the
                // host reads it only every fourth iteration (a host round trip costs more than
                // the few-row launches of an iteration that has nothing left to do)
                if (sync_due_shaped(rt)) {
                    rc = read_count(counts + rcur, &R_host);
                    if (rc) return rc;
                }
            }
            StepShape sh;
            fa.act = cand_list;
            fa.count_dev = counts + 2;
            fa.M_act = k;
            fa.moments_only = true;
            rc = timed(K_REFKURT, 2.0 * n * k * dT, [&] { return run_fused(c, L, fa, &sh); });
            if (rc) return rc;
            KL(launch_kurt_finalize(s, at<float>(c, L.part_mom), sh.splits, sh.part_rows, cand_list, counts + 2, k,
                                    inv_T, alpha, ups));
            KL(launch_argmax(s, ups, nullptr, cand_list, counts + 2, k, slots));
            if (o.record_cands)
                KL(launch_record_cands(s, G, n, N, B32, n_pad, cand, k, o.record_cands + static_cast<int64_t>(i) * k * N));
        }
        if (o.record_features && o.record_labels)
            KL(launch_record(s, traj, itc, B32, n_pad, n, M, slots, std::log(static_cast<double>(T)), uref,
                             o.record_features + static_cast<int64_t>(i) * M * kMlpIn,
                             o.record_labels + static_cast<int64_t>(i) * M));
        // w_i = b_p G appended to W (Algorithm 2)
        rc = timed(K_APPEND, 0.0, [&] {
            KL(launch_append(s, G, n, N, B32, n_pad, slots, alpha, ups, W_out, i, kurt_out + i, cstats + 4 * i));
            if (alg1) KL(launch_w_to_f32(s, W_out, i, N, W32, n_pad));
            return ICA_OK;
        });
        if (rc) return rc;
        comp_iters.push_back(t);
        comp_refine.push_back(rt);
        comp_pruned.push_back(n_pruned);
        comp_fallback.push_back(fell_back);
        comp_kurt_rows.push_back(kurt_rows);
        comp_hist.push_back(hist);
        if (o.profile) {
            CK(cudaStreamSynchronize(s));
            const double before = c->kind_ms[K_ITER];
            harvest(c);
            comp_stage_ms.push_back(c->kind_ms[K_ITER] - before);
            ev_cursor = 0;
        }
        found = i + 1;
        if (o.gauss_test) {
            // Gaussianity test (Eq. 3): the remaining components are Gaussian
            CK(cudaMemcpyAsync(c->host_d, cstats + 4 * i, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(c->host_i + 1, status, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            rc = map_device_status(c->host_i[1]);
            if (rc) return rc;
            const double u_p = c->host_d[2];
            if (u_p < 2.0 * (N - (i + 1) + 2) * (N - (i + 1) + 1) / static_cast<double>(T)) {
                found = i;
                break;
            }
        }
    }
    CK(cudaEventRecord(fit_end, s));
    const int nst = found > 0 ? found : 1;
    CK(cudaMemcpyAsync(c->host_d, cstats, sizeof(double) * 4 * nst, cudaMemcpyDeviceToHost, s));
    std::vector<long long> rows_h(2 * (N + 1));
    CK(cudaMemcpyAsync(rows_h.data(), crows, sizeof(long long) * 2 * (N + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->host_i + 1, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaEventSynchronize(fit_end));
    CK(cudaStreamSynchronize(s));
    float fit_ms = 0.f;
    rc = map_device_status(c->host_i[1]);
    if (rc) return rc;
    CK(cudaEventElapsedTime(&fit_ms, fit_begin, fit_end));
    // algorithmic FLOPs from the exact per-component counts of updated rows (4 n rows T)
    double it_flops = 0.0, ref_flops = 0.0;
    for (int i = 0; i < static_cast<int>(comp_iters.size()); ++i) {
        it_flops += 4.0 * (alg1 ? N : N - i) * static_cast<double>(rows_h[2 * i]) * dT;
        ref_flops += 4.0 * (alg1 ? N : N - i) * static_cast<double>(rows_h[2 * i + 1]) * dT;
    }
    c->kind_flops[K_ITER] = it_flops;
    c->kind_flops[K_REFINE] = ref_flops;
    double kurt_flops = 0.0;
    for (int i = 0; i < static_cast<int>(comp_iters.size()); ++i)
        kurt_flops += 2.0 * (alg1 ? N : N - i) * static_cast<double>(comp_kurt_rows[i]) * dT;
    c->kind_flops[K_KURT] = kurt_flops;
    std::string js = "{\"components\": [";
    for (int i = 0; i < found; ++i) {
        const double p = c->host_d[4 * i], a_p = c->host_d[4 * i + 1], u_p = c->host_d[4 * i + 2];
        if (p < 0) return ICA_ERR_NONFINITE;
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "%s{\"i\": %d, \"iterations\": %d, \"winner\": %d, \"alpha\": %.12g, \"upsilon\": %.12g, "
                 "\"refine_iterations\": %d, \"rows_updated\": %lld, \"refine_rows\": %lld, \"pruned\": %d, "
                 "\"fallback\": %d, \"stage_ms\": %.6f, \"active\": [",
                 i ? ", " : "", i + 1, comp_iters[i], static_cast<int>(p), a_p, u_p, comp_refine[i], rows_h[2 * i],
                 rows_h[2 * i + 1], comp_pruned[i], comp_fallback[i],
                 i < static_cast<int>(comp_stage_ms.size()) ? comp_stage_ms[i] : 0.0);
        js += buf;
        for (size_t h = 0; h < comp_hist[i].size(); ++h) {
            snprintf(buf, sizeof(buf), "%s%d", h ? ", " : "", comp_hist[i][h]);
            js += buf;
        }
        js += "]}";
    }
    js += "], ";
    json_kv(js, "fit_ms", fit_ms);
    json_kv(js, "launches", static_cast<double>(c->launches));
    json_kv(js, "launches_total", static_cast<double>(c->launches_total));
    json_kv(js, "stage_persistent_launches", static_cast<double>(persist_launches));
    json_kv(js, "stage_fp8_launches", static_cast<double>(fp8_launches));
    {   // the persistent stage's first iteration (all M restarts) in equal work shares
        int tl = 0, sp0 = 0, cps0 = 0;
        const int tc0 = tc_chunk(round_up(N, 16));
        const int tot0 = static_cast<int>((T + tc0 - 1) / tc0);
        tc_device_shape(M, 152, tot0, &tl, &sp0, &cps0);
        const bool sk0 = o.stage_streamk && tl * sp0 < (152 * 15) / 16 && static_cast<int64_t>(tl) * tot0 >= 152;
        json_kv(js, "stage_streamk_first_iteration", (persist_launches > 0 && sk0) ? 1.0 : 0.0);
    }
    js += "\"stage_persistent_note\": \"" + c->persist_note + "\", ";
    js += "\"fused\": {";
    for (int k = 0; k < 4; ++k) {
        char buf[200];
        snprintf(buf, sizeof(buf), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e}", k ? ", " : "",
                 kKindName[k], c->kind_n[k], c->kind_ms[k], c->kind_flops[k]);
        js += buf;
    }
    js += "}, \"phases\": {";
    for (int k = 4; k < K_NKINDS; ++k) {
        char buf[160];
        snprintf(buf, sizeof(buf), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f}", k > 4 ? ", " : "", kKindName[k],
                 c->kind_n[k], c->kind_ms[k]);
        js += buf;
    }
    js += "}, ";
    json_kv(js, "n_found", found, false);
    js += "}";
    c->stats = js;
    *n_found = found;
    return ICA_OK;
}

int ica_last_stats(ica_ctx* c, char* buf, size_t cap) {
    if (!c || !buf || cap == 0) return ICA_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    const size_t n = c->stats.size() < cap - 1 ? c->stats.size() : cap - 1;
    memcpy(buf, c->stats.data(), n);
    buf[n] = 0;
    return ICA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Learned restart pruner: network kernels (k_mlp.cu) behind the C ABI.
// ---------------------------------------------------------------------------------------------
static_assert(ICA_MLP_PARAMS == ica::kMlpParams && ICA_MLP_IN == ica::kMlpIn, "pruner layout");

int ica_mlp_init(ica_ctx* c, uint64_t seed, float* params) {
    if (!c || !params) return ICA_ERR_ARG;
    CK(cudaSetDevice(c->device));
    KL(launch_mlp_init(c->stream, seed, params));
    return ICA_OK;
}

int ica_mlp_standardize(ica_ctx* c, const float* F, int rows, float* params) {
    if (!c || !F || !params || rows < 1) return ICA_ERR_ARG;
    CK(cudaSetDevice(c->device));
    KL(launch_mlp_standardize(c->stream, F, rows, params));
    return ICA_OK;
}

int ica_mlp_forward(ica_ctx* c, const float* params, const float* F, int rows, int fp16, float* prob) {
    if (!c || !params || !F || !prob || rows < 1) return ICA_ERR_ARG;
    CK(cudaSetDevice(c->device));
    KL(launch_mlp_forward(c->stream, params, F, rows, fp16 != 0, prob));
    return ICA_OK;
}

size_t ica_mlp_scratch_bytes(int rows) { return rows < 1 ? 0 : mlp_scratch_bytes(rows); }

int ica_mlp_train_step(ica_ctx* c, float* params, float* adam_m, float* adam_v, int step, const float* F,
                       const float* labels, int rows, float lr, float pos_weight, int fp16, void* scratch,
                       size_t scratch_bytes, float* loss, float* grad) {
    if (!c || !params || !adam_m || !adam_v || !F || !labels || rows < 1 || step < 1 || !scratch ||
        !(lr >= 0.f) || !(pos_weight > 0.f))
        return ICA_ERR_ARG;
    if (scratch_bytes < mlp_scratch_bytes(rows)) return ICA_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(scratch) % 16) return ICA_ERR_ARG;
    CK(cudaSetDevice(c->device));
    KL(launch_mlp_train_step(c->stream, params, adam_m, adam_v, step, F, labels, rows, lr, pos_weight, fp16 != 0,
                             static_cast<float*>(scratch), loss, grad));
    c->launches += 2;  // three kernels: forward/backward, gradient slices, Adam
    c->launches_total += 2;
    return ICA_OK;
}

// ---------------------------------------------------------------------------------------------
// Many data sets in one call (ica_order_fit_batched): `workers` fits run concurrently, each on
// a worker context with its own stream and a slice of the caller's workspace; data sets are
// handed to the workers in order from an atomic counter. Before the fits an autotuner picks the
// share of the GPU each fused launch aims for (one wave, a half or a quarter of the SMs) by
// timing concurrent fused steps of a representative data set on all worker streams.
// ---------------------------------------------------------------------------------------------
namespace {
size_t batched_slot_bytes(const ica_dataset* sets, int count, int M, const ica_opts* o) {
    size_t mx = 0;
    for (int k = 0; k < count; ++k) {
        const size_t b = ica_workspace_bytes(sets[k].N, sets[k].T, M, o);
        if (b == 0) return 0;
        if (b > mx) mx = b;
    }
    return align_up(mx);
}

int batched_workers(int count, int workers) {
    int w = workers > 0 ? workers : 8;
    if (w > count) w = count;
    if (w > 32) w = 32;
    return w < 1 ? 1 : w;
}

// Times `reps` concurrent fused update steps (all M rows, zero data: the tensor-core work does
// not depend on the values) on every worker stream for each CTA share; returns the best share.
int autotune_cta_div(ica_ctx* c, int nw, const ica_dataset& rep, int M, int precision, std::vector<float>* times) {
    const int cands[3] = {1, 2, 4};
    const int prec = precision == ICA_PLAIN_FP32 ? ICA_FP32 : precision;
    const int n_pad = round_up(rep.N, 16);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    struct Guard {
        cudaEvent_t a, b;
        ~Guard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } g{e0, e1};
    std::vector<cudaEvent_t> done(nw);
    for (auto& e : done) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    struct Guard2 {
        std::vector<cudaEvent_t>& v;
        ~Guard2() {
            for (auto e : v) cudaEventDestroy(e);
        }
    } g2{done};
    const Layout L = make_layout(rep.N, rep.T, M, prec);
    for (int w = 0; w < nw; ++w) {
        ica_ctx* k = c->workers[w];
        CK(cudaMemsetAsync(k->ws, 0, L.total, k->stream));
    }
    CK(cudaDeviceSynchronize());
    int best = 1;
    float best_ms = 0.f;
    for (int ci = 0; ci < 3; ++ci) {
        CK(cudaEventRecord(e0, c->stream));
        for (int w = 0; w < nw; ++w) {
            ica_ctx* k = c->workers[w];
            k->cta_div = cands[ci];
            CK(cudaStreamWaitEvent(k->stream, e0, 0));
            FusedArgs fa;
            fa.precision = prec;
            fa.B32 = at<float>(k, L.B32);
            fa.ldb = n_pad;
            fa.M_act = M;
            fa.n_pad = n_pad;
            fa.T = rep.T;
            fa.Xt32 = at<float>(k, L.Xt32);
            fa.Xt16 = at<uint16_t>(k, L.Xt16);
            fa.ldx = L.ldx;
            for (int r = 0; r < 3; ++r) {
                StepShape sh;
                const int rc = run_fused(k, L, fa, &sh);
                if (rc) return -rc;
            }
            CK(cudaEventRecord(done[w], k->stream));
            CK(cudaStreamWaitEvent(c->stream, done[w], 0));
        }
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (times) times->push_back(ms);
        if (ci == 0 || ms < best_ms) {
            best_ms = ms;
            best = cands[ci];
        }
    }
    return best;
}
}  // namespace

size_t ica_batched_workspace_bytes(const ica_dataset* sets, int count, int M, const ica_opts* opts, int workers) {
    if (!sets || count < 1 || M < 1) return 0;
    const size_t slot = batched_slot_bytes(sets, count, M, opts);
    return slot ? slot * static_cast<size_t>(batched_workers(count, workers)) : 0;
}

int ica_order_fit_batched(ica_ctx* c, const ica_dataset* sets, int count, int M, int iters, double tol, uint64_t seed,
                          const ica_opts* opts, int workers) {
    if (!c || !sets || count < 1 || M < 1 || M > 65536 || iters < 1 || !(tol > 0.0)) return ICA_ERR_ARG;
    ica_opts d;
    ica_default_opts(&d);
    const ica_opts& o = opts ? *opts : d;
    if (o.B0 || o.record_features || o.record_labels) return ICA_ERR_ARG;  // per-fit buffers have no batched form
    for (int k = 0; k < count; ++k) {
        const ica_dataset& ds = sets[k];
        if (!ds.Xw || !ds.W_out || !ds.kurt_out || !ds.n_found || ds.N < 1 || ds.N > kMaxN ||
            ds.T < 2 * static_cast<int64_t>(ds.N) || ds.n_components < 1 || ds.n_components > ds.N)
            return ICA_ERR_ARG;
    }
    const int nw = batched_workers(count, workers);
    const size_t slot = batched_slot_bytes(sets, count, M, &o);
    if (!slot) return ICA_ERR_ARG;
    if (!c->ws || c->ws_bytes < slot * nw) return ICA_ERR_WORKSPACE;
    CK(cudaSetDevice(c->device));
    while (static_cast<int>(c->workers.size()) < nw) {
        ica_ctx* w = nullptr;
        const int rc = ica_create(&w, c->device);
        if (rc) return rc;
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            ica_destroy(w);
            return ICA_ERR_CUDA;
        }
        w->stream = st;
        c->workers.push_back(w);
        c->worker_streams.push_back(st);
    }
    for (int w = 0; w < nw; ++w) {
        c->workers[w]->ws = c->ws + slot * w;
        c->workers[w]->ws_bytes = slot;
    }
    // representative data set for the autotuner: the median by samples x dimension
    std::vector<int> order(count);
    for (int k = 0; k < count; ++k) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return static_cast<double>(sets[a].N) * sets[a].T < static_cast<double>(sets[b].N) * sets[b].T;
    });
    const ica_dataset& rep = sets[order[count / 2]];
    const long long key = static_cast<long long>(nw) * 1000003LL + round_up(rep.N, 16) * 131LL +
                          static_cast<long long>(std::log2(static_cast<double>(rep.T)));
    int div = 0;
    std::vector<float> tune_ms;
    for (auto& kv : c->tuned)
        if (kv.first == key) div = kv.second;
    if (!div) {
        div = autotune_cta_div(c, nw, rep, M, o.precision, &tune_ms);
        if (div < 0) return -div;
        c->tuned.push_back({key, div});
    }
    // the fits
    cudaEvent_t start;
    CK(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    CK(cudaEventRecord(start, c->stream));
    for (int w = 0; w < nw; ++w) {
        c->workers[w]->cta_div = nw == 1 ? 1 : div;
        if (nw > 1) c->workers[w]->persist_ok = false;
        if (cudaStreamWaitEvent(c->workers[w]->stream, start, 0) != cudaSuccess) {
            cudaEventDestroy(start);
            return ICA_ERR_CUDA;
        }
    }
    cudaEventDestroy(start);
    std::atomic<int> next{0};
    std::vector<int> rcs(count, ICA_OK);
    std::vector<std::string> st(count);
    std::vector<long long> launches(nw, 0);
    std::vector<std::string> errs(count);
    auto t0 = std::chrono::steady_clock::now();
    std::vector<std::thread> pool;
    for (int w = 0; w < nw; ++w) {
        pool.emplace_back([&, w] {
            ica_ctx* k = c->workers[w];
            cudaSetDevice(k->device);
            for (;;) {
                const int i = next.fetch_add(1);
                if (i >= count) break;
                const ica_dataset& ds = sets[i];
                rcs[i] = ica_order_fit(k, ds.Xw, ds.N, ds.T, M, ds.n_components, iters, tol, seed + static_cast<uint64_t>(i),
                                       &o, ds.W_out, ds.kurt_out, ds.n_found);
                st[i] = rcs[i] == ICA_OK ? k->stats : std::string("null");
                if (rcs[i]) errs[i] = g_last_error;
                launches[w] += k->launches;
            }
        });
    }
    for (auto& th : pool) th.join();
    const double wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int w = 0; w < nw; ++w) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        CK(cudaEventRecord(e, c->workers[w]->stream));
        CK(cudaStreamWaitEvent(c->stream, e, 0));
        cudaEventDestroy(e);
    }
    c->launches = 0;
    for (long long l : launches) c->launches += l;
    std::string js = "{\"batched\": {";
    char buf[256];
    snprintf(buf, sizeof(buf), "\"count\": %d, \"workers\": %d, \"cta_div\": %d, \"wall_ms\": %.3f, \"launches\": %lld, \"tune_ms\": [",
             count, nw, div, wall_ms, c->launches);
    js += buf;
    for (size_t k = 0; k < tune_ms.size(); ++k) {
        snprintf(buf, sizeof(buf), "%s%.4f", k ? ", " : "", tune_ms[k]);
        js += buf;
    }
    js += "]}, \"datasets\": [";
    for (int k = 0; k < count; ++k) {
        js += k ? ", " : "";
        js += st[k];
    }
    js += "]}";
    c->stats = js;
    for (int k = 0; k < count; ++k)
        if (rcs[k]) {
            g_last_error = "data set " + std::to_string(k) + ": " + errs[k];
            return rcs[k];
        }
    return ICA_OK;
}

const char* ica_last_error(void) { return g_last_error.c_str(); }
