// FP64 linear algebra on the GPU: whitening statistics (row means, covariance), a one-CTA
// parallel cyclic Jacobi eigensolver for symmetric matrices (m <= 256), and small strided FP64
// products used to form the reduction basis G = (F~F~^T)^(-1/2) F~ of Section 3.3.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace ica {

// ------------------------------------------------------------------------------ row means
// Row means in FP64. A row holding NaN or Inf makes its sum non-finite: DEV_NONFINITE is raised
// (status may be null).
__global__ void __launch_bounds__(256) row_mean_kernel(const float* __restrict__ X, int N, int64_t T, int64_t ld,
                                                       double* __restrict__ mean, int* status) {
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
        if (!isfinite(tot) && status) atomicOr(status, DEV_NONFINITE);
    }
}
cudaError_t launch_row_mean(cudaStream_t s, const float* X, int N, int64_t T, int64_t ld, double* mean, int* status) {
    row_mean_kernel<<<N, 256, 0, s>>>(X, N, T, ld, mean, status);
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
// Only the blocks with a <= b are computed; block (b, a) is written as the transpose, which
// keeps A exactly symmetric and halves the arithmetic on A.
//
// GB300 runs FP64 at 1/64 of the FP32 rate, and one CTA does all of the work, so the
// eigensolver is FP64-bound. For m <= kJacMixedMax it runs in two phases:
//   1. FP32 sweeps on A scaled by a power of two, until the off-diagonal mass is below 1e-11
//      of the total (or 12 sweeps): V32 holds the eigenvectors to ~1e-6;
//   2. FP64 polish: two Newton-Schulz steps V <- V (3I - V^T V) / 2 make V orthogonal to
//      rounding, A' = V^T A V is then diagonal up to ~1e-6, and FP64 sweeps started from
//      (A', V) converge quadratically (two sweeps in practice) to the same stopping rule as the
//      plain FP64 solver.
// The result is an FP64 eigendecomposition (backward stable: V orthogonal to rounding, A = V
// diag(lam) V^T to rounding) at about a third of the FP64 work of FP64 sweeps from the start.
// The four m x m FP64 buffers live in shared memory up to m = kJacSmemMax; above, in a global
// scratch (L2 resident), with the FP32 phase's two m x m matrices still in shared memory up to
// m = kJacF32SmemMax. Smaller m, or calls without a scratch, run FP64 sweeps only.
constexpr int kJacMixedMin = 12, kJacSmemMax = 80, kJacF32SmemMax = 128;

// Pair a of round r in the circle ordering of me = m + (m odd) indices (p < q; q = m is the
// dummy index of odd m). r, a < me - 1 and a <= (me - 1) / 2, so no modulo is needed.
__device__ __forceinline__ void rr_pair(int r, int a, int me, int& p, int& q) {
    const int mm = me - 1;
    if (a == 0) {
        p = r;
        q = mm;
    } else {
        p = r + a;
        if (p >= mm) p -= mm;
        q = r - a;
        if (q < 0) q += mm;
    }
    if (p > q) {
        const int t = p;
        p = q;
        q = t;
    }
}

// Jacobi rotation (c, s) zeroing a_pq (Golub & Van Loan, Algorithm 8.5.1): t is the root of
// smaller magnitude of t^2 + 2 tau t - 1 = 0, tau = (a_qq - a_pp) / (2 a_pq), c = (1+t^2)^-1/2.
__device__ __forceinline__ void rot_params(float apq, float app, float aqq, float& c, float& s) {
    const float tau = (aqq - app) / (2.f * apq);
    const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
    c = 1.f / sqrtf(1.f + t * t);
    s = t * c;
}
// FP64: the FP32 tangent, refined by two Newton steps on f(t) = a_pq t^2 + (a_qq - a_pp) t - a_pq
// (same roots) with an FP32 reciprocal of f'(t) (each step multiplies the relative error by
// about 1e-7), then c by two Newton steps for (1 + t^2)^-1/2 from an FP32 start. Only FP64
// multiply-adds: FP64 division and square root would run on the block's one parameter warp at
// the low FP64 rate of this GPU. Requires entries of order one (the callers scale A).
__device__ __forceinline__ void rot_params(double apq, double app, double aqq, double& c, double& s) {
    const double d = aqq - app;
    const float a32 = static_cast<float>(apq);
    if (a32 == 0.f) {  // |a_pq| < 1e-45 against entries of order one: below rounding
        c = 1.0;
        s = 0.0;
        return;
    }
    float c32, s32;
    rot_params(a32, static_cast<float>(app), static_cast<float>(aqq), c32, s32);
    double t = static_cast<double>(s32 / c32);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double f = fma(fma(apq, t, d), t, -apq);
        const double r = static_cast<double>(1.f / static_cast<float>(fma(2.0 * apq, t, d)));
        t = fma(-f, r, t);
    }
    const double u = fma(t, t, 1.0);
    double y = static_cast<double>(rsqrtf(static_cast<float>(u)));
#pragma unroll
    for (int it = 0; it < 2; ++it) y = y * fma(-0.5 * u, y * y, 1.5);
    c = y;
    s = t * y;
}

// Rotation (c, s) that zeroes A[p][q] for each pair of round r (one thread per pair).
template <typename T>
__device__ __forceinline__ void jac_params(const T* A, int m, int me, int np, int r, T* rc, T* rs) {
    const int tid = threadIdx.x;
    if (tid < np) {
        int p, q;
        rr_pair(r, tid, me, p, q);
        T c = T(1), sn = T(0);
        if (q < m) {
            const T apq = A[p * m + q];
            if (apq != T(0)) rot_params(apq, A[p * m + p], A[q * m + q], c, sn);
        }
        rc[tid] = c;
        rs[tid] = sn;
    }
}

// Per-thread walk over the np x np block indices e = tid, tid + nth, ... as (e / np, e % np),
// advanced without division.
struct BlockWalk {
    int a0, b0, da, db;
    __device__ __forceinline__ BlockWalk(int np) {
        a0 = static_cast<int>(threadIdx.x) / np;
        b0 = static_cast<int>(threadIdx.x) % np;
        da = static_cast<int>(blockDim.x) / np;
        db = static_cast<int>(blockDim.x) % np;
    }
};

// A <- J^T A J (upper blocks, mirrored) and V <- V J for the rotations of round r.
template <typename T>
__device__ __forceinline__ void jac_apply(T* A, T* V, int m, int me, int np, int r, const T* rc, const T* rs,
                                          const BlockWalk& w) {
    const int tid = threadIdx.x, nth = blockDim.x;
    int a = w.a0, b = w.b0;
    for (int e = tid; e < np * np; e += nth) {
        if (a <= b) {
            int pa, qa, pb, qb;
            rr_pair(r, a, me, pa, qa);
            rr_pair(r, b, me, pb, qb);
            const T ca = rc[a], sa = rs[a], cb = rc[b], sb = rs[b];
            const bool qa_ok = qa < m, qb_ok = qb < m;
            const T x00 = A[pa * m + pb];
            const T x01 = qb_ok ? A[pa * m + qb] : T(0);
            const T x10 = qa_ok ? A[qa * m + pb] : T(0);
            const T x11 = (qa_ok && qb_ok) ? A[qa * m + qb] : T(0);
            // rows: (p) c x_p - s x_q, (q) s x_p + c x_q
            const T y00 = ca * x00 - sa * x10, y01 = ca * x01 - sa * x11;
            const T y10 = sa * x00 + ca * x10, y11 = sa * x01 + ca * x11;
            // columns: (p) c y_p - s y_q, (q) s y_p + c y_q
            T z00 = cb * y00 - sb * y01, z01 = sb * y00 + cb * y01;
            T z10 = cb * y10 - sb * y11, z11 = sb * y10 + cb * y11;
            if (a == b) {  // the rotated pair's own block: its off-diagonal is zero by construction
                z01 = T(0);
                z10 = T(0);
            }
            A[pa * m + pb] = z00;
            if (qb_ok) A[pa * m + qb] = z01;
            if (qa_ok) A[qa * m + pb] = z10;
            if (qa_ok && qb_ok) A[qa * m + qb] = z11;
            if (a != b) {  // block (b, a) = block (a, b)^T
                A[pb * m + pa] = z00;
                if (qb_ok) A[qb * m + pa] = z01;
                if (qa_ok) A[pb * m + qa] = z10;
                if (qa_ok && qb_ok) A[qb * m + qa] = z11;
            }
        }
        a += w.da;
        b += w.db;
        if (b >= np) {
            b -= np;
            ++a;
        }
    }
    int i = w.a0;
    b = w.b0;
    for (int e = tid; e < m * np; e += nth) {
        int pb, qb;
        rr_pair(r, b, me, pb, qb);
        if (qb < m) {
            const T cb = rc[b], sb = rs[b];
            const T vp = V[i * m + pb], vq = V[i * m + qb];
            V[i * m + pb] = cb * vp - sb * vq;
            V[i * m + qb] = sb * vp + cb * vq;
        }
        i += w.da;
        b += w.db;
        if (b >= np) {
            b -= np;
            ++i;
        }
    }
}

// Sweeps until off-diagonal mass <= rel_tol * total mass. Returns 1 when converged, 2 when
// max_sweeps sweeps ran without converging, 3 when A holds a non-finite value. Called by
// every thread of the block; the return value is uniform. red holds 64 doubles.
template <typename T>
__device__ int jac_sweeps(T* A, T* V, int m, double rel_tol, int max_sweeps, double* red, int* stop_sh, T* rc,
                          T* rs) {
    const int me = m + (m & 1), np = me / 2;
    const int tid = threadIdx.x, nth = blockDim.x;
    const BlockWalk walk(np);
    for (int sweep = 0;; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = tid; i < m * m; i += nth) {
            const double v = static_cast<double>(A[i]);
            tot += v * v;
            if (i / m != i % m) off += v * v;
        }
        off = warp_sum(off);
        tot = warp_sum(tot);
        if ((tid & 31) == 0) {
            red[tid >> 5] = off;
            red[32 + (tid >> 5)] = tot;
        }
        __syncthreads();
        if (tid == 0) {
            double o = 0.0, t = 0.0;
            for (int i = 0; i < nth / 32; ++i) {
                o += red[i];
                t += red[32 + i];
            }
            int st = 0;
            if (!isfinite(t))
                st = 3;
            else if (o <= rel_tol * t || o == 0.0)
                st = 1;
            else if (sweep >= max_sweeps)
                st = 2;
            *stop_sh = st;
        }
        __syncthreads();
        const int st = *stop_sh;
        __syncthreads();  // red and stop_sh are rewritten by the next sweep
        if (st) return st;
        for (int r = 0; r < me - 1; ++r) {
            jac_params(A, m, me, np, r, rc, rs);
            __syncthreads();
            jac_apply(A, V, m, me, np, r, rc, rs, walk);
            __syncthreads();
        }
    }
}

// Exact power-of-two scale 2^-floor(log2 max|A_ij|) that brings the largest entry into [1, 2)
// (1 for a zero matrix); the rotation parameters assume entries of order one. Called by every
// thread; red holds 64 doubles.
__device__ double jac_scale(const double* Ag, int mm, double* red) {
    const int tid = threadIdx.x, nth = blockDim.x;
    double amax = 0.0;
    for (int i = tid; i < mm; i += nth) amax = fmax(amax, fabs(Ag[i]));
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((tid & 31) == 0) red[tid >> 5] = amax;
    __syncthreads();
    if (tid == 0) {
        double x = 0.0;
        for (int i = 0; i < nth / 32; ++i) x = fmax(x, red[i]);
        red[40] = x;
    }
    __syncthreads();
    amax = red[40];
    __syncthreads();
    if (!(amax > 0.0) || !isfinite(amax)) return 1.0;
    const int e = ilogb(amax);
    return ldexp(1.0, -(e < -1000 ? -1000 : (e > 1000 ? 1000 : e)));
}

// FP64 sweeps from (A, V = I): the solver for m > kJacMixedMax (and tiny m). Stops when the
// off-diagonal mass is below (1e-15)^2 of the total, or after max_sweeps sweeps (then
// DEV_ILLCOND is raised). A is read from its upper triangle.
__global__ void __launch_bounds__(1024) jacobi_kernel(double* Ag, double* Vg, double* lam, int m, int* status,
                                                      int max_sweeps, int use_smem) {
    extern __shared__ double jsm[];
    __shared__ double rc[kMaxN / 2], rs[kMaxN / 2];
    __shared__ double red[64];
    __shared__ int stop;
    double* A = use_smem ? jsm : Ag;
    double* V = use_smem ? jsm + m * m : Vg;
    const int tid = threadIdx.x, nth = blockDim.x;
    const double scale = jac_scale(Ag, m * m, red), unscale = 1.0 / scale;  // powers of two: exact
    for (int i = tid; i < m * m; i += nth) {  // upper triangle scaled (each entry by its own thread)
        const int r = i / m, c = i % m;
        if (r <= c) A[i] = Ag[i] * scale;
        V[i] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int i = tid; i < m * m; i += nth) {  // mirrored into the lower triangle
        const int r = i / m, c = i % m;
        if (r > c) A[i] = A[c * m + r];
    }
    __syncthreads();
    const int st = jac_sweeps<double>(A, V, m, 1e-30, max_sweeps, red, &stop, rc, rs);
    if (st >= 2 && tid == 0) atomicOr(status, DEV_ILLCOND);
    for (int i = tid; i < m; i += nth) lam[i] = A[i * m + i] * unscale;
    __syncthreads();  // A may be Ag itself: unscale in place only after the diagonal was read
    for (int i = tid; i < m * m; i += nth) {
        Ag[i] = A[i] * unscale;
        if (use_smem) Vg[i] = V[i];
    }
}

// Symmetric product C = X^T Y of m x m shared-memory matrices when X^T Y is known to be
// symmetric (upper triangle computed, mirrored), or general C = X Y (sym = false, transA =
// false). Called by every thread; ends with a barrier.
__device__ __forceinline__ void jac_gemm(const double* X, const double* Y, double* C, int m, bool transA, bool sym) {
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int e = tid; e < m * m; e += nth) {
        const int r = e / m, c = e % m;
        if (sym && r > c) continue;
        double acc = 0.0;
        if (transA)
            for (int k = 0; k < m; ++k) acc = fma(X[k * m + r], Y[k * m + c], acc);
        else
            for (int k = 0; k < m; ++k) acc = fma(X[r * m + k], Y[k * m + c], acc);
        C[e] = acc;
        if (sym && r != c) C[c * m + r] = acc;
    }
    __syncthreads();
}

// Mixed-precision solver for m >= kJacMixedMin (see above). Four m x m FP64 buffers P0..P3: in
// shared memory (gP null; the FP32 phase keeps its A and V in P2 and P3), or at gP (4 m^2
// doubles) with the FP32 A and V in shared memory (f32_smem) or at gP32 (2 m^2 floats).
__global__ void __launch_bounds__(1024) jacobi_mixed_kernel(double* Ag, double* Vg, double* lam, int m, int* status,
                                                            int max_sweeps, double* gP, float* gP32, int f32_smem) {
    extern __shared__ double jsm[];
    __shared__ double rcd[kMaxN / 2], rsd[kMaxN / 2];
    __shared__ float rcf[kMaxN / 2], rsf[kMaxN / 2];
    __shared__ double red[64];
    __shared__ int stop;
    const int mm = m * m;
    const int tid = threadIdx.x, nth = blockDim.x;
    double* base = gP ? gP : jsm;
    double* P0 = base;  // A (FP64, kept)
    double* P1 = base + mm;
    double* P2 = base + 2 * mm;
    double* P3 = base + 3 * mm;
    float* A32 = !gP ? reinterpret_cast<float*>(P2) : (f32_smem ? reinterpret_cast<float*>(jsm) : gP32);
    float* V32 = !gP ? reinterpret_cast<float*>(P3) : (f32_smem ? reinterpret_cast<float*>(jsm) + mm : gP32 + mm);
    const double scale = jac_scale(Ag, mm, red), unscale = 1.0 / scale;  // powers of two: exact
    for (int i = tid; i < mm; i += nth) {
        const int r = i / m, c = i % m;
        const double v = (r <= c ? Ag[i] : Ag[c * m + r]) * scale;
        P0[i] = v;
        A32[i] = static_cast<float>(v);
        V32[i] = (r == c) ? 1.f : 0.f;
    }
    __syncthreads();
    int st = jac_sweeps<float>(A32, V32, m, 1e-11, 12, red, &stop, rcf, rsf);
    if (st == 3) {  // non-finite input: report it, return A's diagonal and V = I
        if (tid == 0) atomicOr(status, DEV_ILLCOND);
        for (int i = tid; i < m; i += nth) lam[i] = P0[i * m + i] * unscale;
        for (int i = tid; i < mm; i += nth) Vg[i] = (i / m == i % m) ? 1.0 : 0.0;
        return;
    }
    for (int i = tid; i < mm; i += nth) P1[i] = static_cast<double>(V32[i]);
    __syncthreads();
    // two Newton-Schulz steps toward the orthogonal polar factor of V
    for (int it = 0; it < 2; ++it) {
        jac_gemm(P1, P1, P2, m, true, true);  // S = V^T V
        for (int e = tid; e < mm; e += nth) {  // V (3I - S) / 2
            const int r = e / m, c = e % m;
            double acc = 0.0;
            for (int k = 0; k < m; ++k) acc = fma(P1[r * m + k], (k == c ? 3.0 : 0.0) - P2[k * m + c], acc);
            P3[e] = 0.5 * acc;
        }
        __syncthreads();
        double* t = P1;
        P1 = P3;
        P3 = t;
    }
    jac_gemm(P0, P1, P2, m, false, false);  // A V
    jac_gemm(P1, P2, P3, m, true, true);    // A' = V^T A V
    st = jac_sweeps<double>(P3, P1, m, 1e-30, max_sweeps, red, &stop, rcd, rsd);
    if (st >= 2 && tid == 0) atomicOr(status, DEV_ILLCOND);
    for (int i = tid; i < m; i += nth) lam[i] = P3[i * m + i] * unscale;
    for (int i = tid; i < mm; i += nth) {
        Ag[i] = P3[i] * unscale;
        Vg[i] = P1[i];
    }
}

size_t jacobi_scratch_bytes(int m) {
    return m > kJacSmemMax ? 4ull * m * m * sizeof(double) + 2ull * m * m * sizeof(float) : 0;
}

cudaError_t launch_jacobi(cudaStream_t s, double* A, double* V, double* lam, int m, int* status, int max_sweeps,
                          void* scratch) {
    int threads = m * m / 2;
    threads = threads < 128 ? 128 : (threads > 1024 ? 1024 : round_up(threads, 32));
    if (m >= kJacMixedMin && (m <= kJacSmemMax || scratch)) {
        const bool in_smem = m <= kJacSmemMax;
        const bool f32_smem = !in_smem && m <= kJacF32SmemMax;
        double* gP = in_smem ? nullptr : static_cast<double*>(scratch);
        float* gP32 = in_smem || f32_smem ? nullptr : reinterpret_cast<float*>(gP + 4ull * m * m);
        const size_t smem = in_smem ? 4ull * m * m * sizeof(double) : (f32_smem ? 2ull * m * m * sizeof(float) : 0);
        cudaError_t e = allow_max_dyn_smem(jacobi_mixed_kernel);
        if (e != cudaSuccess) return e;
        jacobi_mixed_kernel<<<1, threads, smem, s>>>(A, V, lam, m, status, max_sweeps, gP, gP32, f32_smem ? 1 : 0);
        return cudaGetLastError();
    }
    const size_t smem = 2ull * m * m * sizeof(double);
    const int use_smem = smem <= 160 * 1024;
    if (use_smem) {
        cudaError_t e = allow_max_dyn_smem(jacobi_kernel);
        if (e != cudaSuccess) return e;
    }
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
