// Reduction of signals (Section 3.3, Eq. 8): X~ = G X, and the whitening apply
// Xw = V X - V mean. FP64 coefficients are rounded to FP32 on load; products accumulate in
// FP32. Writes FP32 rows and/or their BF16 rounding (the tensor-core operand). Rows n..n_pad-1
// are written as zeros, so the padded reduced dimension contributes nothing to the products.
#include "common.cuh"
#include "internal.h"

namespace ica {

constexpr int RG_BM = 64, RG_BT = 128, RG_BK = 16;

__global__ void __launch_bounds__(256) rows_gemm_kernel(const double* __restrict__ G, int n, int N,
                                                        const float* __restrict__ X, int64_t T, int64_t ldxin,
                                                        const double* __restrict__ bias, float* __restrict__ out32,
                                                        int64_t ld32, uint16_t* __restrict__ out16, int64_t ld16,
                                                        int n_pad) {
    __shared__ __align__(16) float Gs[RG_BK][RG_BM + 4];  // padded: the transposing stores spread over banks
    __shared__ __align__(16) float Xs[RG_BK][RG_BT];
    const int rb = blockIdx.x, tb = blockIdx.y;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t t0 = static_cast<int64_t>(tb) * RG_BT;
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    const bool vec_ok = (ldxin % 4 == 0);
    for (int k0 = 0; k0 < N; k0 += RG_BK) {
        for (int e = threadIdx.x; e < RG_BK * RG_BM; e += 256) {  // a row's 16 coefficients per 16 threads
            const int rr = e / RG_BK, kk = e % RG_BK;
            const int r = rb * RG_BM + rr, k = k0 + kk;
            Gs[kk][rr] = (r < n && k < N) ? static_cast<float>(G[static_cast<int64_t>(r) * N + k]) : 0.f;
        }
        for (int e = threadIdx.x; e < RG_BK * (RG_BT / 4); e += 256) {
            const int kk = e / (RG_BT / 4), c4 = (e % (RG_BT / 4)) * 4;
            const int k = k0 + kk;
            const int64_t t = t0 + c4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < N) {
                const float* src = X + static_cast<int64_t>(k) * ldxin + t;
                if (vec_ok && t + 3 < T) {
                    v = *reinterpret_cast<const float4*>(src);
                } else {
                    if (t < T) v.x = src[0];
                    if (t + 1 < T) v.y = src[1];
                    if (t + 2 < T) v.z = src[2];
                    if (t + 3 < T) v.w = src[3];
                }
            }
            *reinterpret_cast<float4*>(&Xs[kk][c4]) = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < RG_BK; ++kk) {
            const float4 g = *reinterpret_cast<const float4*>(&Gs[kk][ty * 4]);
            // samples tx*4.. and 64 + tx*4..: consecutive threads read consecutive 16-byte words
            const float4 xa = *reinterpret_cast<const float4*>(&Xs[kk][tx * 4]);
            const float4 xb = *reinterpret_cast<const float4*>(&Xs[kk][RG_BT / 2 + tx * 4]);
            const float gv[4] = {g.x, g.y, g.z, g.w};
            const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(gv[i], xv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = rb * RG_BM + ty * 4 + i;
        const float b = (bias && r < n) ? static_cast<float>(bias[r]) : 0.f;
        float v[8];  // samples tx*4 + j (j < 4) and 64 + tx*4 + (j - 4)
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = r < n ? acc[i][j] - b : 0.f;
        if (r >= n_pad) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const float* vh = v + 4 * half;
            const int64_t t = t0 + half * (RG_BT / 2) + tx * 4;
            if (out32) {
                float* dst = out32 + static_cast<int64_t>(r) * ld32 + t;
                if (t + 3 < T && (ld32 % 4 == 0)) {
                    *reinterpret_cast<float4*>(dst) = make_float4(vh[0], vh[1], vh[2], vh[3]);
                } else {
                    for (int j = 0; j < 4; ++j)
                        if (t + j < T) dst[j] = vh[j];
                }
            }
            if (out16) {
                uint16_t* dst = out16 + static_cast<int64_t>(r) * ld16 + t;
                if (t + 3 < T && (ld16 % 4 == 0)) {
                    uint2 pk;
                    pk.x = pack_bf16x2(vh[0], vh[1]);
                    pk.y = pack_bf16x2(vh[2], vh[3]);
                    *reinterpret_cast<uint2*>(dst) = pk;
                } else {
                    for (int j = 0; j < 4; ++j)
                        if (t + j < T) dst[j] = static_cast<uint16_t>(pack_bf16x2(vh[j], 0.f) & 0xffffu);
                }
            }
        }
    }
}

cudaError_t launch_rows_gemm(cudaStream_t s, const double* G, int n, int n_pad, int N, const float* X, int64_t T,
                             int64_t ldxin, const double* bias, float* out32, int64_t ld32, uint16_t* out16,
                             int64_t ld16) {
    dim3 grid((n_pad + RG_BM - 1) / RG_BM, static_cast<unsigned>((T + RG_BT - 1) / RG_BT));
    rows_gemm_kernel<<<grid, 256, 0, s>>>(G, n, N, X, T, ldxin, bias, out32, ld32, out16, ld16, n_pad);
    return cudaGetLastError();
}


// ------------------------------------------------------------------------------------------
// E4M3 copy of X~ for the FP8 stage iterations. Row k is stored as e4m3(x~ 2^e_k) with the
// power-of-two scale 2^e_k that maps the row's largest magnitude into the format's range
// (|.| <= 448); padding rows and samples are zero. sc receives, per row k < n_pad,
// sc[k] = 2^e_k, sc[n_pad + k] = 2^(c - e_k) (the scale of the restart rows' column k, with
// c = 8 + min_k e_k so that unit-norm rows stay within 2^8), sc[2 n_pad + k] = 2^-e_k, and
// sc[3 n_pad] = 2^-c (the first product's output -> z).
// ------------------------------------------------------------------------------------------
namespace {

__global__ void __launch_bounds__(256) row_absmax_kernel(const float* __restrict__ X, int64_t ldx, int64_t T,
                                                         unsigned* __restrict__ rmax) {
    __shared__ float wm[8];
    const int k = blockIdx.y;
    const float* row = X + static_cast<int64_t>(k) * ldx;
    float m = 0.f;
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x * 4;
    for (int64_t t = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 4; t < T; t += step) {
        if (t + 3 < T) {
            const float4 v = *reinterpret_cast<const float4*>(row + t);
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        } else {
            for (int j = 0; j < 4; ++j)
                if (t + j < T) m = fmaxf(m, fabsf(row[t + j]));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, wm[w]);
        atomicMax(rmax + k, __float_as_uint(m));  // non-negative floats order as their bit patterns
    }
}

__global__ void fp8_scales_kernel(const unsigned* __restrict__ rmax, int n, int n_pad, float* __restrict__ sc) {
    __shared__ int emin;
    const int k = threadIdx.x;
    const int e = k < n ? pow2_fit_exponent(__uint_as_float(rmax[k]), 448.f) : 0;
    if (k == 0) emin = 1 << 20;
    __syncthreads();
    if (k < n) atomicMin(&emin, e);
    __syncthreads();
    const int c = 8 + (n > 0 ? emin : 0);
    if (k < n_pad) {
        sc[k] = ldexpf(1.f, e);
        sc[n_pad + k] = ldexpf(1.f, c - e);
        sc[2 * n_pad + k] = ldexpf(1.f, -e);
    }
    if (k == 0) sc[3 * n_pad] = ldexpf(1.f, -c);
}

__global__ void __launch_bounds__(256) to_e4m3_kernel(const float* __restrict__ X, int64_t ldx, int64_t T, int n,
                                                      const float* __restrict__ sc, uint8_t* __restrict__ X8,
                                                      int64_t ld8) {
    const int k = blockIdx.y;
    const float s = k < n ? sc[k] : 0.f;
    const float* row = X + static_cast<int64_t>(k) * ldx;
    uint8_t* dst = X8 + static_cast<int64_t>(k) * ld8;
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x * 16;
    for (int64_t t = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 16; t < ld8; t += step) {
        float v[16];
        if (k < n && t + 15 < T) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 q = *reinterpret_cast<const float4*>(row + t + 4 * i);
                v[4 * i] = q.x * s;
                v[4 * i + 1] = q.y * s;
                v[4 * i + 2] = q.z * s;
                v[4 * i + 3] = q.w * s;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = (k < n && t + i < T) ? row[t + i] * s : 0.f;
        }
        uint4 w;
        w.x = pack_e4m3x4(v[0], v[1], v[2], v[3]);
        w.y = pack_e4m3x4(v[4], v[5], v[6], v[7]);
        w.z = pack_e4m3x4(v[8], v[9], v[10], v[11]);
        w.w = pack_e4m3x4(v[12], v[13], v[14], v[15]);
        *reinterpret_cast<uint4*>(dst + t) = w;
    }
}

}  // namespace

cudaError_t launch_fp8_copy(cudaStream_t s, const float* X32, int64_t ldx, int64_t T, int n, int n8,
                            unsigned* rmax, float* sc, uint8_t* X8, int64_t ld8, int* launches) {
    if (n8 > 256 || n > n8 || ld8 % 16 != 0 || ld8 < T) return cudaErrorInvalidValue;
    const int n_pad = n8;
    cudaError_t e = cudaMemsetAsync(rmax, 0, sizeof(unsigned) * n_pad, s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        const int64_t bx = (T + 1023) / 1024;
        row_absmax_kernel<<<dim3(static_cast<unsigned>(bx < 64 ? bx : 64), n), 256, 0, s>>>(X32, ldx, T, rmax);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    fp8_scales_kernel<<<1, 256, 0, s>>>(rmax, n, n_pad, sc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t cx = (ld8 / 16 + 255) / 256;
    to_e4m3_kernel<<<dim3(static_cast<unsigned>(cx < 128 ? cx : 128), n_pad), 256, 0, s>>>(X32, ldx, T, n, sc, X8, ld8);
    if (launches) *launches += n > 0 ? 3 : 2;
    return cudaGetLastError();
}

}  // namespace ica
