// Fused FP32 iteration of the matrix form (Section 3.1; Algorithm 2 update) on CUDA cores:
// for a tile of 64 active restarts and a contiguous sample range, Z = B X~ chunk by chunk in
// registers, Z o Z o Z staged in shared memory, and acc += (Z o Z o Z) X~^T kept in
// registers; Z never reaches device memory. Also accumulates sum z^2, sum z^4 (and
// sum (z^2 - 1)^2 in the moments-only variant used for the kurtosis of candidates).
// Outputs are per-split partial sums, reduced in a fixed order by the finalize kernels.
#include "common.cuh"
#include "internal.h"

namespace ica {

constexpr int F_MT = kFp32Rows;  // restart rows per CTA
constexpr int F_TC = 64;         // samples per chunk
constexpr int F_XS = F_TC + 4;   // padded row stride of the X~ chunk in shared memory

size_t fp32_smem_bytes(int n_pad) {
    return sizeof(float) * (static_cast<size_t>(n_pad) * F_MT + static_cast<size_t>(n_pad) * F_XS +
                            static_cast<size_t>(F_TC) * F_MT);
}

template <bool MOMENTS_ONLY>
__global__ void __launch_bounds__(256) fused_fp32_kernel(const float* __restrict__ B32, int ldb,
                                                         const int* __restrict__ act_idx,
                                                         const int* __restrict__ count_dev, int M_act_host,
                                                         const float* __restrict__ Xt, int64_t ldx, int n_pad,
                                                         int64_t T, int chunks_per_split, float* __restrict__ part_acc,
                                                         float* __restrict__ part_mom, int part_rows) {
    extern __shared__ __align__(16) float fsm[];
    float* Bs = fsm;                   // [n_pad][F_MT]  (k-major, restart contiguous)
    float* Xs = Bs + n_pad * F_MT;     // [n_pad][F_XS]
    float* Zs = Xs + n_pad * F_XS;     // [F_TC][F_MT]   (z^3, sample-major; 16-byte groups of
                                       // restarts XOR-swizzled by sample/4 against bank conflicts)
    const int split = blockIdx.x, tile = blockIdx.y;
    const int m0 = tile * F_MT;
    const int M_act = count_dev ? *count_dev : M_act_host;
    if (m0 >= M_act) return;  // grid sized for an upper bound of the active count
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int kj = n_pad / 16;

    for (int e = tid; e < n_pad * F_MT; e += 256) {
        const int k = e / F_MT, m = e % F_MT;
        const int gm = m0 + m;
        float v = 0.f;
        if (gm < M_act) {
            const int r = act_idx ? act_idx[gm] : gm;
            v = B32[static_cast<int64_t>(r) * ldb + k];
        }
        Bs[k * F_MT + m] = v;
    }

    const int64_t c_begin = static_cast<int64_t>(split) * chunks_per_split;
    const int64_t total_chunks = (T + F_TC - 1) / F_TC;
    const int64_t c_end = c_begin + chunks_per_split < total_chunks ? c_begin + chunks_per_split : total_chunks;

    float acc[4][16];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[i][j] = 0.f;
    float m2[4] = {0.f, 0.f, 0.f, 0.f}, m4[4] = {0.f, 0.f, 0.f, 0.f}, mq[4] = {0.f, 0.f, 0.f, 0.f};

    for (int64_t c = c_begin; c < c_end; ++c) {
        const int64_t t0 = c * F_TC;
        __syncthreads();  // previous chunk fully consumed (and B tile written on the first pass)
        for (int e = tid; e < n_pad * (F_TC / 4); e += 256) {
            const int k = e / (F_TC / 4), c4 = (e % (F_TC / 4)) * 4;
            const int64_t t = t0 + c4;
            const float* src = Xt + static_cast<int64_t>(k) * ldx + t;
            float4 v;
            if (t + 3 < T) {
                v = *reinterpret_cast<const float4*>(src);
            } else {
                v.x = t < T ? src[0] : 0.f;
                v.y = t + 1 < T ? src[1] : 0.f;
                v.z = t + 2 < T ? src[2] : 0.f;
                v.w = t + 3 < T ? src[3] : 0.f;
            }
            *reinterpret_cast<float4*>(&Xs[k * F_XS + c4]) = v;
        }
        __syncthreads();
        // Z tile: rows ty*4..+4, samples tx*4..+4
        float z[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) z[i][j] = 0.f;
        for (int k = 0; k < n_pad; ++k) {
            const float4 b = *reinterpret_cast<const float4*>(&Bs[k * F_MT + ty * 4]);
            const float4 x = *reinterpret_cast<const float4*>(&Xs[k * F_XS + tx * 4]);
            const float bv[4] = {b.x, b.y, b.z, b.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) z[i][j] = fmaf(bv[i], xv[j], z[i][j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool valid = t0 + tx * 4 + j < T;
            float z3[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float zz = z[i][j], z2 = zz * zz;
                m2[i] += z2;
                m4[i] = fmaf(z2, z2, m4[i]);
                z3[i] = z2 * zz;
                if (MOMENTS_ONLY) {
                    const float e = valid ? z2 - 1.f : 0.f;
                    mq[i] = fmaf(e, e, mq[i]);
                }
            }
            if (!MOMENTS_ONLY) {
                const int t = tx * 4 + j;
                *reinterpret_cast<float4*>(&Zs[t * F_MT + ((ty ^ ((t >> 2) & 15)) << 2)]) =
                    make_float4(z3[0], z3[1], z3[2], z3[3]);
            }
        }
        if (!MOMENTS_ONLY) {
            __syncthreads();
            for (int t = 0; t < F_TC; ++t) {
                const float4 zc = *reinterpret_cast<const float4*>(&Zs[t * F_MT + ((ty ^ ((t >> 2) & 15)) << 2)]);
                const float zv[4] = {zc.x, zc.y, zc.z, zc.w};
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (j >= kj) break;  // uniform exit: no predicated-off work for small n
                    const float x = Xs[(tx + 16 * j) * F_XS + t];
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[i][j] = fmaf(zv[i], x, acc[i][j]);
                }
            }
        }
    }
    // moments: reduce over the 16 sample lanes (tx) sharing a restart row
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            m2[i] += __shfl_xor_sync(0xffffffffu, m2[i], o);
            m4[i] += __shfl_xor_sync(0xffffffffu, m4[i], o);
            mq[i] += __shfl_xor_sync(0xffffffffu, mq[i], o);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = m0 + ty * 4 + i;
        if (row >= M_act) continue;
        const int64_t prow = static_cast<int64_t>(split) * part_rows + row;
        if (tx == 0) {
            part_mom[prow * 4 + 0] = m2[i];
            part_mom[prow * 4 + 1] = m4[i];
            part_mom[prow * 4 + 2] = mq[i];
            part_mom[prow * 4 + 3] = 0.f;
        }
        if (!MOMENTS_ONLY) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if (j >= kj) break;
                part_acc[prow * n_pad + tx + 16 * j] = acc[i][j];
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Small-batch variant for at most 16 restart rows (the FP32 refinement of a few distinct
// candidates): one row per thread row, 16 rows x 64 samples per chunk, so no tensor work is
// spent on empty rows and the launch is bound by reading X~ once.
// ------------------------------------------------------------------------------------------
constexpr int S_MT = 16;
constexpr int S_ZS = S_MT + 1;  // padded z^3 row stride (bank conflicts)

size_t fp32_small_smem_bytes(int n_pad) {
    return sizeof(float) * (static_cast<size_t>(S_MT) * n_pad + static_cast<size_t>(n_pad) * F_XS +
                            static_cast<size_t>(F_TC) * S_ZS);
}

template <bool MOMENTS_ONLY>
__global__ void __launch_bounds__(256) fused_fp32_small_kernel(const float* __restrict__ B32, int ldb,
                                                               const int* __restrict__ act_idx,
                                                               const int* __restrict__ count_dev, int M_act_host,
                                                               const float* __restrict__ Xt, int64_t ldx, int n_pad,
                                                               int64_t T, int chunks_per_split,
                                                               float* __restrict__ part_acc,
                                                               float* __restrict__ part_mom, int part_rows) {
    extern __shared__ __align__(16) float ssm[];
    float* Bs = ssm;                  // [S_MT][n_pad]
    float* Xs = Bs + S_MT * n_pad;    // [n_pad][F_XS]
    float* Zs = Xs + n_pad * F_XS;    // [F_TC][S_ZS]
    const int M_act = count_dev ? *count_dev : M_act_host;
    const int split = blockIdx.x;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // ty = restart row, tx = sample group
    const int kj = n_pad / 16;
    for (int e = tid; e < S_MT * n_pad; e += 256) {
        const int m = e / n_pad, k = e % n_pad;
        float v = 0.f;
        if (m < M_act) {
            const int r = act_idx ? act_idx[m] : m;
            v = B32[static_cast<int64_t>(r) * ldb + k];
        }
        Bs[e] = v;
    }
    const int64_t c_begin = static_cast<int64_t>(split) * chunks_per_split;
    const int64_t total_chunks = (T + F_TC - 1) / F_TC;
    const int64_t c_end = c_begin + chunks_per_split < total_chunks ? c_begin + chunks_per_split : total_chunks;
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.f;
    float m2 = 0.f, m4 = 0.f, mq = 0.f;
    for (int64_t c = c_begin; c < c_end; ++c) {
        const int64_t t0 = c * F_TC;
        __syncthreads();
        for (int e = tid; e < n_pad * (F_TC / 4); e += 256) {
            const int k = e / (F_TC / 4), c4 = (e % (F_TC / 4)) * 4;
            const int64_t t = t0 + c4;
            const float* src = Xt + static_cast<int64_t>(k) * ldx + t;
            float4 v;
            if (t + 3 < T) {
                v = *reinterpret_cast<const float4*>(src);
            } else {
                v.x = t < T ? src[0] : 0.f;
                v.y = t + 1 < T ? src[1] : 0.f;
                v.z = t + 2 < T ? src[2] : 0.f;
                v.w = t + 3 < T ? src[3] : 0.f;
            }
            *reinterpret_cast<float4*>(&Xs[k * F_XS + c4]) = v;
        }
        __syncthreads();
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < n_pad; ++k) {
            const float b = Bs[ty * n_pad + k];
            const float4 x = *reinterpret_cast<const float4*>(&Xs[k * F_XS + tx * 4]);
            z[0] = fmaf(b, x.x, z[0]);
            z[1] = fmaf(b, x.y, z[1]);
            z[2] = fmaf(b, x.z, z[2]);
            z[3] = fmaf(b, x.w, z[3]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float z2 = z[j] * z[j];
            m2 += z2;
            m4 = fmaf(z2, z2, m4);
            if (MOMENTS_ONLY) {
                const float e = (t0 + tx * 4 + j < T) ? z2 - 1.f : 0.f;
                mq = fmaf(e, e, mq);
            } else {
                Zs[(tx * 4 + j) * S_ZS + ty] = z2 * z[j];
            }
        }
        if (!MOMENTS_ONLY) {
            __syncthreads();
            for (int t = 0; t < F_TC; ++t) {
                const float zc = Zs[t * S_ZS + ty];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (j >= kj) break;  // uniform exit: no predicated-off work for small n
                    acc[j] = fmaf(zc, Xs[(tx + 16 * j) * F_XS + t], acc[j]);
                }
            }
        }
    }
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        m4 += __shfl_xor_sync(0xffffffffu, m4, o);
        mq += __shfl_xor_sync(0xffffffffu, mq, o);
    }
    if (ty >= M_act) return;
    const int64_t prow = static_cast<int64_t>(split) * part_rows + ty;
    if (tx == 0) {
        part_mom[prow * 4 + 0] = m2;
        part_mom[prow * 4 + 1] = m4;
        part_mom[prow * 4 + 2] = mq;
        part_mom[prow * 4 + 3] = 0.f;
    }
    if (!MOMENTS_ONLY) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j >= kj) break;
            part_acc[prow * n_pad + tx + 16 * j] = acc[j];
        }
    }
}

cudaError_t launch_fused_fp32_small(cudaStream_t s, bool moments_only, const float* B32, int ldb, const int* act_idx,
                                    const int* count_dev, int M_act_host, const float* Xt, int64_t ldx, int n_pad,
                                    int64_t T, int splits, int chunks_per_split, float* part_acc, float* part_mom,
                                    int part_rows) {
    const size_t smem = fp32_small_smem_bytes(n_pad);
    cudaError_t e;
    if (moments_only) {
        e = cudaFuncSetAttribute(fused_fp32_small_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        fused_fp32_small_kernel<true><<<splits, 256, smem, s>>>(B32, ldb, act_idx, count_dev, M_act_host, Xt, ldx,
                                                                n_pad, T, chunks_per_split, part_acc, part_mom,
                                                                part_rows);
    } else {
        e = cudaFuncSetAttribute(fused_fp32_small_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        fused_fp32_small_kernel<false><<<splits, 256, smem, s>>>(B32, ldb, act_idx, count_dev, M_act_host, Xt, ldx,
                                                                 n_pad, T, chunks_per_split, part_acc, part_mom,
                                                                 part_rows);
    }
    return cudaGetLastError();
}

cudaError_t launch_fused_fp32(cudaStream_t s, bool moments_only, const float* B32, int ldb, const int* act_idx,
                              const int* count_dev, int M_act, const float* Xt, int64_t ldx, int n_pad, int64_t T,
                              int splits, int chunks_per_split, float* part_acc, float* part_mom, int part_rows) {
    const size_t smem = fp32_smem_bytes(n_pad);
    const dim3 grid(splits, (M_act + F_MT - 1) / F_MT);
    cudaError_t e;
    if (moments_only) {
        e = cudaFuncSetAttribute(fused_fp32_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        fused_fp32_kernel<true><<<grid, 256, smem, s>>>(B32, ldb, act_idx, count_dev, M_act, Xt, ldx, n_pad, T,
                                                        chunks_per_split, part_acc, part_mom, part_rows);
    } else {
        e = cudaFuncSetAttribute(fused_fp32_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        fused_fp32_kernel<false><<<grid, 256, smem, s>>>(B32, ldb, act_idx, count_dev, M_act, Xt, ldx, n_pad, T,
                                                         chunks_per_split, part_acc, part_mom, part_rows);
    }
    return cudaGetLastError();
}

}  // namespace ica
