// FP64 linear algebra on the GPU: whitening statistics (row means, covariance), a one-CTA
// parallel cyclic Jacobi eigensolver for symmetric matrices (m <= 256), and small strided FP64
// products used to form the reduction basis G = (F~F~^T)^(-1/2) F~ of Section 3.3.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace ica {

// ------------------------------------------------------------------------------ row means
__global__ void __launch_bounds__(256) row_mean_kernel(const float* __restrict__ X, int N, int64_t T, int64_t ld,
                                                       double* __restrict__ mean) {
    __shared__ double red[8];
    const int r = blockIdx.x;
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < T; t += 256) s += static_cast<double>(X[r * ld + t]);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < 8; ++i) tot += red[i];
        mean[r] = tot / static_cast<double>(T);
    }
}
cudaError_t launch_row_mean(cudaStream_t s, const float* X, int N, int64_t T, int64_t ld, double* mean) {
    row_mean_kernel<<<N, 256, 0, s>>>(X, N, T, ld, mean);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ covariance
// C = (X - mean)(X - mean)^T / T in FP64. CTA (tile pair, split): a 32x32 tile of C over a
// contiguous sample range; only tiles on or above the diagonal are computed. Partial tiles are
// written per split and summed in a fixed order by cov_reduce_kernel (deterministic).
constexpr int CV_TILE = 32, CV_TC = 64;

__global__ void __launch_bounds__(256) cov_partial_kernel(const float* __restrict__ X, const double* __restrict__ mean,
                                                          int N, int64_t T, int64_t ld, int64_t per_split,
                                                          double* __restrict__ part) {
    __shared__ double As[CV_TILE][CV_TC + 1];
    __shared__ double Bs[CV_TILE][CV_TC + 1];
    const int nt = (N + CV_TILE - 1) / CV_TILE;
    int tile = blockIdx.x, ti = 0;
    while (tile >= nt - ti) {  // map linear index to (ti, tj) with tj >= ti
        tile -= nt - ti;
        ++ti;
    }
    const int tj = ti + tile;
    const int split = blockIdx.y;
    const int64_t t_begin = split * per_split, t_end = min(T, t_begin + per_split);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t t0 = t_begin; t0 < t_end; t0 += CV_TC) {
        for (int e = threadIdx.x; e < CV_TILE * CV_TC; e += 256) {
            const int rr = e / CV_TC, cc = e % CV_TC;
            const int64_t t = t0 + cc;
            const int ra = ti * CV_TILE + rr, rb = tj * CV_TILE + rr;
            As[rr][cc] = (ra < N && t < t_end) ? static_cast<double>(X[ra * ld + t]) - mean[ra] : 0.0;
            Bs[rr][cc] = (rb < N && t < t_end) ? static_cast<double>(X[rb * ld + t]) - mean[rb] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int c = 0; c < CV_TC; ++c) {
            const double a0 = As[ty * 2][c], a1 = As[ty * 2 + 1][c];
            const double b0 = Bs[tx * 2][c], b1 = Bs[tx * 2 + 1][c];
            acc[0][0] += a0 * b0;
            acc[0][1] += a0 * b1;
            acc[1][0] += a1 * b0;
            acc[1][1] += a1 * b1;
        }
        __syncthreads();
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const int r = ti * CV_TILE + ty * 2 + i, c = tj * CV_TILE + tx * 2 + j;
            if (r < N && c < N) part[(static_cast<int64_t>(split) * N + r) * N + c] = acc[i][j];
        }
}

__global__ void cov_reduce_kernel(const double* __restrict__ part, int splits, int N, double inv_T,
                                  double* __restrict__ C) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * N) return;
    const int r = i / N, c = i % N;
    const int rr = r <= c ? r : c, cc = r <= c ? c : r;  // partials exist on/above the diagonal tiles
    const int tr = rr / CV_TILE, tc = cc / CV_TILE;
    int src_r = rr, src_c = cc;
    if (tr == tc) {  // diagonal tile holds both triangles
        src_r = r;
        src_c = c;
    }
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += part[(static_cast<int64_t>(sp) * N + src_r) * N + src_c];
    C[i] = s * inv_T;
}

int covariance_splits(int N, int64_t T) {
    const int nt = (N + CV_TILE - 1) / CV_TILE;
    const int tiles = nt * (nt + 1) / 2;
    int splits = (2 * 152 + tiles - 1) / tiles;
    const int64_t max_by_T = (T + 1023) / 1024;
    if (splits > max_by_T) splits = static_cast<int>(max_by_T);
    if (splits < 1) splits = 1;
    return splits;
}

cudaError_t launch_covariance(cudaStream_t s, const float* X, const double* mean, int N, int64_t T, int64_t ld,
                              double* part, int splits, double* C) {
    const int nt = (N + CV_TILE - 1) / CV_TILE;
    const int tiles = nt * (nt + 1) / 2;
    const int64_t per = round_up64((T + splits - 1) / splits, CV_TC);
    cov_partial_kernel<<<dim3(tiles, splits), 256, 0, s>>>(X, mean, N, T, ld, per, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cov_reduce_kernel<<<(N * N + 255) / 256, 256, 0, s>>>(part, splits, N, 1.0 / static_cast<double>(T), C);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ Jacobi
// Two-sided cyclic Jacobi (Golub & Van Loan, Matrix Computations, Sec. 8.5) with the
// round-robin (circle) ordering: every round applies m/2 disjoint rotations at once, so a
// round updates each 2x2 block (pair a, pair b) of A independently: A <- J^T A J, V <- V J.
// A (m x m, ld m) is overwritten; on exit lam[i] = A[i][i] and the columns of V are the
// eigenvectors. Stops when the off-diagonal mass is below (1e-15)^2 of the total, or after
// max_sweeps sweeps (then DEV_ILLCOND is raised). The matrices live in shared memory when
// they fit, else in global memory (L2 resident).
__device__ __forceinline__ void rr_pair(int r, int a, int me, int& p, int& q) {
    const int mm = me - 1;
    if (a == 0) {
        p = r;
        q = mm;
    } else {
        p = (r + a) % mm;
        q = (r - a + mm) % mm;
    }
    if (p > q) {
        const int t = p;
        p = q;
        q = t;
    }
}

__global__ void __launch_bounds__(1024) jacobi_kernel(double* Ag, double* Vg, double* lam, int m, int* status,
                                                      int max_sweeps, int use_smem) {
    extern __shared__ double jsm[];
    __shared__ double rc[kMaxN / 2], rs[kMaxN / 2];
    __shared__ double red[32];
    __shared__ int stop;
    const int me = m + (m & 1);
    const int np = me / 2;
    double* A = use_smem ? jsm : Ag;
    double* V = use_smem ? jsm + m * m : Vg;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < m * m; i += nth) {
        if (use_smem) A[i] = Ag[i];
        V[i] = (i / m == i % m) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0;; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = tid; i < m * m; i += nth) {
            const double v = A[i];
            tot += v * v;
            if (i / m != i % m) off += v * v;
        }
        off = warp_sum(off);
        tot = warp_sum(tot);
        if ((tid & 31) == 0) {
            red[tid >> 5] = off;
        }
        __syncthreads();
        if (tid == 0) {
            double o = 0.0;
            for (int i = 0; i < nth / 32; ++i) o += red[i];
            red[31] = o;
        }
        __syncthreads();
        const double off_all = red[31];
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = tot;
        __syncthreads();
        if (tid == 0) {
            double o = 0.0;
            for (int i = 0; i < nth / 32; ++i) o += red[i];
            stop = (off_all <= 1e-30 * o) || (off_all == 0.0);
            if (!stop && sweep >= max_sweeps) {
                atomicOr(status, DEV_ILLCOND);
                stop = 1;
            }
        }
        __syncthreads();
        if (stop) break;
        for (int r = 0; r < me - 1; ++r) {
            if (tid < np) {
                int p, q;
                rr_pair(r, tid, me, p, q);
                double c = 1.0, sn = 0.0;
                if (q < m) {
                    const double apq = A[p * m + q];
                    if (apq != 0.0) {
                        const double app = A[p * m + p], aqq = A[q * m + q];
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = t * c;
                    }
                }
                rc[tid] = c;
                rs[tid] = sn;
            }
            __syncthreads();
            // A <- J^T A J on every 2x2 block (pair a rows, pair b columns)
            for (int e = tid; e < np * np; e += nth) {
                const int a = e / np, b = e % np;
                int pa, qa, pb, qb;
                rr_pair(r, a, me, pa, qa);
                rr_pair(r, b, me, pb, qb);
                const double ca = rc[a], sa = rs[a], cb = rc[b], sb = rs[b];
                const bool qa_ok = qa < m, qb_ok = qb < m;
                const double x00 = A[pa * m + pb];
                const double x01 = qb_ok ? A[pa * m + qb] : 0.0;
                const double x10 = qa_ok ? A[qa * m + pb] : 0.0;
                const double x11 = (qa_ok && qb_ok) ? A[qa * m + qb] : 0.0;
                // rows: (p) c x_p - s x_q, (q) s x_p + c x_q
                const double y00 = ca * x00 - sa * x10, y01 = ca * x01 - sa * x11;
                const double y10 = sa * x00 + ca * x10, y11 = sa * x01 + ca * x11;
                // columns: (p) c y_p - s y_q, (q) s y_p + c y_q
                double z00 = cb * y00 - sb * y01, z01 = sb * y00 + cb * y01;
                double z10 = cb * y10 - sb * y11, z11 = sb * y10 + cb * y11;
                if (a == b) {  // the rotated pair's own block: its off-diagonal is zero by construction
                    z01 = 0.0;
                    z10 = 0.0;
                }
                A[pa * m + pb] = z00;
                if (qb_ok) A[pa * m + qb] = z01;
                if (qa_ok) A[qa * m + pb] = z10;
                if (qa_ok && qb_ok) A[qa * m + qb] = z11;
            }
            // V <- V J
            for (int e = tid; e < m * np; e += nth) {
                const int i = e / np, b = e % np;
                int pb, qb;
                rr_pair(r, b, me, pb, qb);
                if (qb >= m) continue;
                const double cb = rc[b], sb = rs[b];
                const double vp = V[i * m + pb], vq = V[i * m + qb];
                V[i * m + pb] = cb * vp - sb * vq;
                V[i * m + qb] = sb * vp + cb * vq;
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < m; i += nth) lam[i] = A[i * m + i];
    if (use_smem)
        for (int i = tid; i < m * m; i += nth) {
            Ag[i] = A[i];
            Vg[i] = V[i];
        }
}

cudaError_t launch_jacobi(cudaStream_t s, double* A, double* V, double* lam, int m, int* status, int max_sweeps) {
    const size_t smem = 2ull * m * m * sizeof(double);
    const int use_smem = smem <= 160 * 1024;
    if (use_smem) {
        cudaError_t e = allow_max_dyn_smem(jacobi_kernel);
        if (e != cudaSuccess) return e;
    }
    int threads = m * m / 2;
    threads = threads < 128 ? 128 : (threads > 1024 ? 1024 : round_up(threads, 32));
    jacobi_kernel<<<1, threads, use_smem ? smem : 0, s>>>(A, V, lam, m, status, max_sweeps, use_smem);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ FP64 products
// C[i][j] = alpha * sum_l A(i,l) B(l,j) + beta * C[i][j], A(i,l) = A[i*sar + l*sac],
// B(l,j) = B[l*sbr + j*sbc]. 16x16 output tile per CTA, inner dimension staged by 16.
__global__ void __launch_bounds__(256) gemm_f64_kernel(int rows, int cols, int inner, double alpha,
                                                       const double* __restrict__ A, int64_t sar, int64_t sac,
                                                       const double* __restrict__ B, int64_t sbr, int64_t sbc,
                                                       double beta, double* __restrict__ C, int64_t ldc) {
    __shared__ double As[16][17], Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
    double acc = 0.0;
    for (int l0 = 0; l0 < inner; l0 += 16) {
        const int ai = blockIdx.y * 16 + ty, al = l0 + tx;
        As[ty][tx] = (ai < rows && al < inner) ? A[ai * sar + al * sac] : 0.0;
        const int bl = l0 + ty, bj = blockIdx.x * 16 + tx;
        Bs[ty][tx] = (bl < inner && bj < cols) ? B[bl * sbr + bj * sbc] : 0.0;
        __syncthreads();
#pragma unroll
        for (int l = 0; l < 16; ++l) acc += As[ty][l] * Bs[l][tx];
        __syncthreads();
    }
    if (i < rows && j < cols) {
        const double old = beta != 0.0 ? C[i * ldc + j] : 0.0;
        C[i * ldc + j] = alpha * acc + beta * old;
    }
}

cudaError_t launch_gemm_f64(cudaStream_t s, int rows, int cols, int inner, double alpha, const double* A,
                            int64_t sar, int64_t sac, const double* B, int64_t sbr, int64_t sbc, double beta,
                            double* C, int64_t ldc) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((cols + 15) / 16, (rows + 15) / 16);
    gemm_f64_kernel<<<grid, 256, 0, s>>>(rows, cols, inner, alpha, A, sar, sac, B, sbr, sbc, beta, C, ldc);
    return cudaGetLastError();
}

__global__ void set_identity_kernel(double* A, int rows, int cols, int64_t ld, double diag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int r = i / cols, c = i % cols;
    A[r * ld + c] = (r == c) ? diag : 0.0;
}
cudaError_t launch_set_identity(cudaStream_t s, double* A, int rows, int cols, int64_t ld, double diag) {
    set_identity_kernel<<<(rows * cols + 255) / 256, 256, 0, s>>>(A, rows, cols, ld, diag);
    return cudaGetLastError();
}

// out[i][j] = Q[i][j] * f(lam[j]) for an m x m eigenvector matrix (columns = eigenvectors).
// fn 0: f = lam^(-1/2)                      (inverse square root)
// fn 1: f = 1 / (s (1 + s)), s = sqrt(1 - lam)  (= ((1 - lam)^(-1/2) - 1) / lam, no cancellation)
// Raises DEV_ILLCOND when fn 0 meets lam <= ill_thresh * max(lam) or fn 1 meets
// 1 - lam <= ill_thresh.
__global__ void scale_cols_fn_kernel(const double* __restrict__ Q, const double* __restrict__ lam, int m, int fn,
                                     double* __restrict__ out, int* status, double ill_thresh) {
    __shared__ double lmax;
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int j = 0; j < m; ++j) mx = fmax(mx, lam[j]);
        lmax = mx;
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * m) return;
    const int j = i % m;
    const double l = lam[j];
    double f;
    if (fn == 0) {
        if (!(l > ill_thresh * lmax)) {
            atomicOr(status, DEV_ILLCOND);
            f = 0.0;
        } else {
            f = 1.0 / sqrt(l);
        }
    } else {
        const double om = 1.0 - l;
        if (!(om > ill_thresh)) {
            atomicOr(status, DEV_ILLCOND);
            f = 0.0;
        } else {
            const double sq = sqrt(om);
            f = 1.0 / (sq * (1.0 + sq));
        }
    }
    out[i] = Q[i] * f;
}
cudaError_t launch_scale_cols_fn(cudaStream_t s, const double* Q, const double* lam, int m, int fn, double* out,
                                 int* status, double ill_thresh) {
    scale_cols_fn_kernel<<<(m * m + 255) / 256, 256, 0, s>>>(Q, lam, m, fn, out, status, ill_thresh);
    return cudaGetLastError();
}

__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ x, double b,
                             const double* __restrict__ y, double* __restrict__ out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + (b != 0.0 ? b * y[i] : 0.0);
}
cudaError_t launch_axpby_f64(cudaStream_t s, int64_t n, double a, const double* x, double b, const double* y,
                             double* out) {
    axpby_kernel<<<static_cast<int>((n + 255) / 256), 256, 0, s>>>(n, a, x, b, y, out);
    return cudaGetLastError();
}

// out (k x N) = W with columns >= ncols zeroed.
__global__ void pad_cols_kernel(const double* __restrict__ W, int k, int N, int ncols, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k * N) return;
    out[i] = (i % N) < ncols ? W[i] : 0.0;
}
cudaError_t launch_pad_cols(cudaStream_t s, const double* W, int k, int N, int ncols, double* out) {
    pad_cols_kernel<<<(k * N + 255) / 256, 256, 0, s>>>(W, k, N, ncols, out);
    return cudaGetLastError();
}

}  // namespace ica
