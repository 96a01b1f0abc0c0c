// Allocation-free variant of the fused update step (ica_fp_step).
//
// Some callers cannot call cudaMalloc: code embedded in an application whose allocator has
// reserved the whole device up front (a framework's caching allocator or an inference
// server's memory pool), plug-ins that may not allocate after start-up, and latency-critical
// loops that must not pay for the implicit device synchronisation cudaFree performs. They still
// own their inputs and outputs but cannot hand this library a workspace. For them this file
// keeps the split-T partial sums of the fused update in a file-scope device array of fixed size
// that every GPU loading the library holds until the process exits.
//
// The array's name is only meaningful in device code; host code must use the address that
// cudaGetSymbolAddress returns for the current device, which is looked up once per device on
// the first call made with that device current.
#include <mutex>

#include "common.cuh"
#include "ica.h"
#include "internal.h"

using namespace ica;

namespace {
constexpr size_t kNoallocScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr size_t kStatusBytes = 256;                        // device status word, padded
constexpr int kMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_fp_step_scratch[kNoallocScratchBytes];

namespace {

typedef CUresult (*PFN_encode_noalloc_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                         const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                         CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                         CUtensorMapFloatOOBfill);

std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};
PFN_encode_noalloc_t g_encode = nullptr;

// Once per device, with that device current: the device address of the scratch array.
int scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ICA_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_fp_step_scratch) != cudaSuccess || !p) return ICA_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    if (!g_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_encode_noalloc_t>(fn);
    }
    *out = g_scratch_addr[dev];
    return ICA_OK;
}

// Split of the sample range with the rule ica_fp_step uses, then capped so that
// splits * part_rows * (n_pad + 4) floats fit in the scratch. one_wave (the BF16 kernel, which
// holds all 512 TMEM columns and so runs one CTA per SM): at most target_ctas CTAs, never a
// partial second wave; otherwise about target_ctas CTAs, rounded up.
int splits_within(int64_t total_chunks, int tiles, int part_rows, int n_pad, int target_ctas, bool one_wave,
                  int* splits, int* cps) {
    const size_t per_split = sizeof(float) * static_cast<size_t>(part_rows) * (n_pad + 4);
    const size_t cap = (kNoallocScratchBytes - kStatusBytes) / per_split;
    if (cap < 1) return ICA_ERR_WORKSPACE;
    int64_t s = one_wave ? (tiles <= target_ctas ? target_ctas / tiles : 1) : (target_ctas + tiles - 1) / tiles;
    const int64_t cta_cap = kMaxCTAs / tiles > 0 ? kMaxCTAs / tiles : 1;
    if (s > cta_cap) s = cta_cap;
    if (s > static_cast<int64_t>(cap)) s = static_cast<int64_t>(cap);
    if (s > total_chunks) s = total_chunks;
    if (s < 1) s = 1;
    const int64_t c = (total_chunks + s - 1) / s;
    *cps = static_cast<int>(c);
    *splits = static_cast<int>((total_chunks + c - 1) / c);
    return ICA_OK;
}

}  // namespace

extern "C" int ica_fp_step_noalloc(int precision, const float* B, int M, int n, const void* Xt, int64_t T,
                                   int64_t ldx, float* Bnew, float* moments, void* stream) {
    if (!B || !Xt || !Bnew || M < 1 || M > 65536 || n < 1 || n > kMaxN || T < 1 || ldx < T || ldx % 8)
        return ICA_ERR_ARG;
    if (precision != ICA_FP32 && precision != ICA_BF16) return ICA_ERR_UNSUPPORTED;
    const int n_pad = round_up(n, 16);
    const bool bf16 = precision == ICA_BF16;
    // the kernel and launch shape ica_fp_step takes for these sizes: 128-row tcgen05 tiles in one
    // wave (BF16), the few-row FP32 kernel for at most kFp32SmallRows rows, 64-row FP32 tiles
    const bool few_rows = !bf16 && M <= kFp32SmallRows;
    const int rows_per_tile = bf16 ? kTcRows : (few_rows ? fp32_rows_tile(M) : kFp32Rows);
    const int tiles = (M + rows_per_tile - 1) / rows_per_tile;
    const int chunk = bf16 ? tc_chunk(n_pad) : (few_rows ? fp32_rows_chunk(n_pad) : 64);
    const int64_t total = (T + chunk - 1) / chunk;
    const int part_rows = tiles * rows_per_tile;
    int splits = 1, cps = 1;
    int rc = splits_within(total, tiles, part_rows, n_pad, bf16 ? 152 : (few_rows ? 2 * 152 : 4 * 152), bf16,
                           &splits, &cps);
    if (rc) return rc;  // one split of M * (n_pad + 4) * 4 bytes does not fit in the 16 MiB scratch
    unsigned char* base = nullptr;
    rc = scratch_for_current_device(&base);
    if (rc) return rc;
    if (bf16 && !g_encode) return ICA_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* status = reinterpret_cast<int*>(base);
    float* part_mom = reinterpret_cast<float*>(base + kStatusBytes);
    float* part_acc = part_mom + static_cast<size_t>(splits) * part_rows * 4;
    // the status word keeps the previous call's value: clear it (the partials are overwritten)
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return ICA_ERR_CUDA;
    cudaError_t e;
    if (bf16) {
        CUtensorMap map;
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(T), static_cast<cuuint64_t>(n_pad)};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldx) * 2};
        cuuint32_t box[2] = {64u, static_cast<cuuint32_t>(n_pad)};
        cuuint32_t estr[2] = {1u, 1u};
        if (g_encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(Xt), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return ICA_ERR_CUDA;
        e = launch_fused_tc(s, false, true, map, B, n_pad, nullptr, nullptr, M, n_pad, T, splits, cps,
                            static_cast<int>(total), part_acc, part_mom, part_rows, status);
    } else if (few_rows) {
        e = launch_fused_fp32_rows(s, false, B, n_pad, nullptr, nullptr, M, static_cast<const float*>(Xt), ldx, n_pad,
                                   T, splits, cps, part_acc, part_mom, part_rows);
    } else {
        e = launch_fused_fp32(s, false, B, n_pad, nullptr, nullptr, M, static_cast<const float*>(Xt), ldx, n_pad, T,
                              splits, cps, part_acc, part_mom, part_rows);
    }
    if (e != cudaSuccess) return ICA_ERR_CUDA;
    if (launch_combine(s, part_acc, part_mom, splits, part_rows, n_pad, M, B, 1.0 / static_cast<double>(T), Bnew,
                       moments) != cudaSuccess)
        return ICA_ERR_CUDA;
    int host_status = 0;
    if (cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ICA_ERR_CUDA;
    if (host_status & DEV_TIMEOUT) return ICA_ERR_TIMEOUT;
    if (host_status & DEV_NONFINITE) return ICA_ERR_NONFINITE;
    return ICA_OK;
}
