// Elementwise kernels of the plain FP32 matrix form (Algorithm 2 written literally, Z = B X~
// materialised in device memory). This path is the comparison baseline for the fused
// kernels; its two products run in cuBLAS SGEMM (FP32, no TF32).
#include "common.cuh"
#include "internal.h"

namespace ica {

// out (M_act x n_pad) = rows act_idx[j] of B32 for j < *count_dev, zero rows beyond (the
// products then run on an upper bound of the active count).
__global__ void gather_rows_kernel(const float* __restrict__ B32, int ldb, const int* __restrict__ act_idx,
                                   const int* __restrict__ count_dev, int M_act, int n_pad, float* __restrict__ out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= static_cast<int64_t>(M_act) * n_pad) return;
    const int count = count_dev ? *count_dev : M_act;
    const int j = static_cast<int>(i / n_pad), k = static_cast<int>(i % n_pad);
    if (j >= count) {
        out[i] = 0.f;
        return;
    }
    const int r = act_idx ? act_idx[j] : j;
    out[i] = B32[static_cast<int64_t>(r) * ldb + k];
}
cudaError_t launch_gather_rows(cudaStream_t s, const float* B32, int ldb, const int* act_idx, const int* count_dev,
                               int M_act, int n_pad, float* out) {
    const int64_t n = static_cast<int64_t>(M_act) * n_pad;
    gather_rows_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(B32, ldb, act_idx, count_dev, M_act,
                                                                              n_pad, out);
    return cudaGetLastError();
}

// Z <- Z o Z o Z (element-wise cube, in place).
__global__ void cube_kernel(float* __restrict__ Z, int rows, int64_t T, int64_t ldz) {
    const int r = blockIdx.y;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < T;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float z = Z[r * ldz + t];
        Z[r * ldz + t] = z * z * z;
    }
}
cudaError_t launch_cube_inplace(cudaStream_t s, float* Z, int rows, int64_t T, int64_t ldz) {
    const int bx = static_cast<int>(((T + 255) / 256) < 64 ? ((T + 255) / 256) : 64);
    cube_kernel<<<dim3(bx, rows), 256, 0, s>>>(Z, rows, T, ldz);
    return cudaGetLastError();
}

// part_mom[r] = (sum z^2, sum z^4, sum (z^2 - 1)^2, 0) over the T samples of row r of Z.
__global__ void __launch_bounds__(256) row_moments_kernel(const float* __restrict__ Z, int rows, int64_t T,
                                                          int64_t ldz, float* __restrict__ part_mom) {
    __shared__ double red[3][8];
    const int r = blockIdx.x;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t t = threadIdx.x; t < T; t += 256) {
        const float z = Z[r * ldz + t];
        const float z2 = z * z;
        a += z2;
        b += static_cast<double>(z2) * z2;
        const float e = z2 - 1.f;
        c += static_cast<double>(e) * e;
    }
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = a;
        red[1][w] = b;
        red[2][w] = c;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += red[threadIdx.x][i];
        part_mom[static_cast<int64_t>(r) * 4 + threadIdx.x] = static_cast<float>(s);
    }
    if (threadIdx.x == 3) part_mom[static_cast<int64_t>(r) * 4 + 3] = 0.f;
}
cudaError_t launch_row_moments(cudaStream_t s, const float* Z, int rows, int64_t T, int64_t ldz, float* part_mom) {
    row_moments_kernel<<<rows, 256, 0, s>>>(Z, rows, T, ldz, part_mom);
    return cudaGetLastError();
}

}  // namespace ica
