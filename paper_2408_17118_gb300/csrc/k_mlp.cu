// Learned restart pruner (not part of the paper's method): a 13-64-64-1 perceptron that reads
// the first five iterations of a restart (kurtosis alpha of Eq. 2 and the step distance of the
// convergence test), n, log T and the gap of the restart's Upsilon (Eq. 1) at iteration 5 to the
// best restart still running then, and predicts whether the restart ends at the direction the
// component picks. Inference and training run here: FP16 weights and activations (the "fp16"
// switch; 0 keeps everything FP32 for gradient checks), FP32 accumulation, FP32 master weights
// and Adam moments.
//
// Parameter vector (FP32, kMlpParams floats): mean[13], scale[13], W1[64][13], b1[64],
// W2[64][64], b2[64], w3[64], b3. Training scratch: per sample a row of kActRow floats
// (x_hat 13, h1 64, d1 64, h2 64, d2 64, dz 1), sample-major, so that the gradient kernel reads
// the activations of one sample with coalesced loads.
#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

namespace ica {

namespace {
constexpr int IN = kMlpIn, HID = kMlpHid;
constexpr int OFF_MEAN = 0, OFF_SCALE = IN, OFF_W1 = 2 * IN, OFF_B1 = OFF_W1 + HID * IN, OFF_W2 = OFF_B1 + HID,
              OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID;
static_assert(OFF_B3 + 1 == kMlpParams, "parameter layout");
constexpr int A_X = 0, A_H1 = IN, A_D1 = A_H1 + HID, A_H2 = A_D1 + HID, A_D2 = A_H2 + HID, A_DZ = A_D2 + HID;
static_assert(A_DZ + 1 <= kActRow, "activation row");

// Rounds to FP16 and back when the kernel runs in FP16 mode.
template <bool H>
__device__ __forceinline__ float q(float x) {
    if constexpr (H) return __half2float(__float2half_rn(x));
    return x;
}

// Weights (rounded in FP16 mode) in shared memory, shared by a block.
struct SmemNet {
    float w1[HID * IN], b1[HID], w2[HID * HID], b2[HID], w3[HID], b3, mean[IN], scale[IN];
};

template <bool H>
__device__ void load_net(const float* __restrict__ p, SmemNet& s) {
    for (int i = threadIdx.x; i < HID * HID; i += blockDim.x) s.w2[i] = q<H>(p[OFF_W2 + i]);
    for (int i = threadIdx.x; i < HID * IN; i += blockDim.x) s.w1[i] = q<H>(p[OFF_W1 + i]);
    for (int i = threadIdx.x; i < HID; i += blockDim.x) {
        s.b1[i] = q<H>(p[OFF_B1 + i]);
        s.b2[i] = q<H>(p[OFF_B2 + i]);
        s.w3[i] = q<H>(p[OFF_W3 + i]);
    }
    if (threadIdx.x < IN) {
        s.mean[threadIdx.x] = p[OFF_MEAN + threadIdx.x];
        s.scale[threadIdx.x] = p[OFF_SCALE + threadIdx.x];
    }
    if (threadIdx.x == 0) s.b3 = q<H>(p[OFF_B3]);
    __syncthreads();
}

// Forward pass of one sample; h1 and h2 (post-ReLU) optionally written to act.
template <bool H>
__device__ float forward_one(const SmemNet& s, const float* x_raw, float* x_hat, float* act) {
    float x[IN];
#pragma unroll
    for (int i = 0; i < IN; ++i) {
        x[i] = q<H>((x_raw[i] - s.mean[i]) * s.scale[i]);
        if (x_hat) x_hat[i] = x[i];
    }
    float h1[HID];
#pragma unroll
    for (int j = 0; j < HID; ++j) {
        float a = s.b1[j];
#pragma unroll
        for (int i = 0; i < IN; ++i) a = fmaf(s.w1[j * IN + i], x[i], a);
        h1[j] = q<H>(fmaxf(a, 0.f));
        if (act) act[A_H1 + j] = h1[j];
    }
    float z = s.b3;
#pragma unroll 4
    for (int k = 0; k < HID; ++k) {
        float a = s.b2[k];
#pragma unroll
        for (int j = 0; j < HID; ++j) a = fmaf(s.w2[k * HID + j], h1[j], a);
        const float h2 = q<H>(fmaxf(a, 0.f));
        if (act) act[A_H2 + k] = h2;
        z = fmaf(s.w3[k], h2, z);
    }
    return z;
}

__device__ __forceinline__ float sigmoidf(float z) { return 1.f / (1.f + __expf(-z)); }

template <bool H>
__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ params, const float* __restrict__ F,
                                                          int rows, float* __restrict__ prob) {
    __shared__ SmemNet s;
    load_net<H>(params, s);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float xr[IN];
#pragma unroll
    for (int i = 0; i < IN; ++i) xr[i] = F[static_cast<int64_t>(r) * IN + i];
    prob[r] = sigmoidf(forward_one<H>(s, xr, nullptr, nullptr));
}

// Forward + backward of one sample per thread: writes its activation row and its loss term.
template <bool H>
__global__ void __launch_bounds__(128) mlp_train_fwd_kernel(const float* __restrict__ params, const float* __restrict__ F,
                                                            const float* __restrict__ y, int rows, float pos_weight,
                                                            float* __restrict__ act, float* __restrict__ loss_part) {
    __shared__ SmemNet s;
    __shared__ float red[128];
    load_net<H>(params, s);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    float lterm = 0.f;
    if (r < rows) {
        float* a = act + static_cast<int64_t>(r) * kActRow;
        float xr[IN];
#pragma unroll
        for (int i = 0; i < IN; ++i) xr[i] = F[static_cast<int64_t>(r) * IN + i];
        const float z = forward_one<H>(s, xr, a + A_X, a);
        const float p = sigmoidf(z);
        const float yy = y[r];
        // -[w y log p + (1 - y) log(1 - p)] with log p = -softplus(-z), log(1 - p) = -softplus(z)
        const float sp_neg = fmaxf(-z, 0.f) + log1pf(__expf(-fabsf(z)));
        const float sp_pos = fmaxf(z, 0.f) + log1pf(__expf(-fabsf(z)));
        lterm = pos_weight * yy * sp_neg + (1.f - yy) * sp_pos;
        const float dz = (p * (pos_weight * yy + 1.f - yy) - pos_weight * yy) / static_cast<float>(rows);
        a[A_DZ] = dz;
        float d2[HID];
#pragma unroll
        for (int k = 0; k < HID; ++k) {
            d2[k] = a[A_H2 + k] > 0.f ? dz * s.w3[k] : 0.f;
            a[A_D2 + k] = d2[k];
        }
#pragma unroll 4
        for (int j = 0; j < HID; ++j) {
            float g = 0.f;
#pragma unroll
            for (int k = 0; k < HID; ++k) g = fmaf(d2[k], s.w2[k * HID + j], g);
            a[A_D1 + j] = a[A_H1 + j] > 0.f ? g : 0.f;
        }
    }
    red[threadIdx.x] = lterm;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// Gradient of every learnable parameter over a slice of the samples (deterministic order).
__global__ void mlp_grad_kernel(const float* __restrict__ act, int rows, int slice, float* __restrict__ gpart) {
    const int pidx = blockIdx.x * blockDim.x + threadIdx.x;  // learnable index 0 .. kMlpParams-25
    if (pidx >= kMlpParams - 2 * IN) return;
    const int P = pidx + 2 * IN;
    int ua, ub;  // activation columns multiplied (ub < 0: bias, the factor is 1)
    if (P < OFF_B1) {
        ua = A_D1 + (P - OFF_W1) / IN;
        ub = A_X + (P - OFF_W1) % IN;
    } else if (P < OFF_W2) {
        ua = A_D1 + (P - OFF_B1);
        ub = -1;
    } else if (P < OFF_B2) {
        ua = A_D2 + (P - OFF_W2) / HID;
        ub = A_H1 + (P - OFF_W2) % HID;
    } else if (P < OFF_W3) {
        ua = A_D2 + (P - OFF_B2);
        ub = -1;
    } else if (P < OFF_B3) {
        ua = A_DZ;
        ub = A_H2 + (P - OFF_W3);
    } else {
        ua = A_DZ;
        ub = -1;
    }
    const int s0 = blockIdx.y * slice, s1 = min(rows, s0 + slice);
    float g = 0.f;
    for (int r = s0; r < s1; ++r) {
        const float* a = act + static_cast<int64_t>(r) * kActRow;
        g = fmaf(a[ua], ub >= 0 ? a[ub] : 1.f, g);
    }
    gpart[static_cast<int64_t>(blockIdx.y) * kMlpParams + P] = g;
}

// Sum of the slices (fixed order), optional copy of the gradient, Adam update; the loss is the
// fixed-order sum of the per-block parts divided by rows.
__global__ void mlp_adam_kernel(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ gpart, int slices, int step, float lr,
                                float* __restrict__ grad_out, const float* __restrict__ loss_part, int nparts, int rows,
                                float* __restrict__ loss_out) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P == 0 && loss_out) {
        float l = 0.f;
        for (int i = 0; i < nparts; ++i) l += loss_part[i];
        *loss_out = l / static_cast<float>(rows);
    }
    if (P >= kMlpParams) return;
    float g = 0.f;
    if (P >= 2 * IN)
        for (int sl = 0; sl < slices; ++sl) g += gpart[static_cast<int64_t>(sl) * kMlpParams + P];
    if (grad_out) grad_out[P] = g;
    if (lr <= 0.f || P < 2 * IN) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mm = b1 * m[P] + (1.f - b1) * g;
    const float vv = b2 * v[P] + (1.f - b2) * g * g;
    m[P] = mm;
    v[P] = vv;
    const float mh = mm / (1.f - powf(b1, static_cast<float>(step)));
    const float vh = vv / (1.f - powf(b2, static_cast<float>(step)));
    params[P] -= lr * mh / (sqrtf(vh) + eps);
}

// He initialisation from Philox4x32-10 (key = seed): W ~ N(0, 2 / fan_in), biases 0, mean 0,
// scale 1.
__global__ void mlp_init_kernel(uint64_t seed, float* __restrict__ params) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= kMlpParams) return;
    float v = 0.f;
    float fan = 0.f;
    if (P >= OFF_SCALE && P < OFF_W1) v = 1.f;
    if (P >= OFF_W1 && P < OFF_B1) fan = IN;
    if (P >= OFF_W2 && P < OFF_B2) fan = HID;
    if (P >= OFF_W3 && P < OFF_B3) fan = HID;
    if (fan > 0.f) {
        const uint4 c = philox4x32_10(make_uint4(static_cast<uint32_t>(P), 0x6d6c70u, 0u, 0u),
                                      make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
        const double u1 = uniform52(c.x, c.y), u2 = uniform52(c.z, c.w);
        const double g = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
        v = static_cast<float>(g * sqrt(2.0 / fan));
    }
    params[P] = v;
}

// Feature standardisation from a set of feature rows: one block per column, fixed order.
__global__ void mlp_standardize_kernel(const float* __restrict__ F, int rows, float* __restrict__ params) {
    __shared__ double red[256];
    const int c = blockIdx.x;
    double sacc = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) sacc += F[static_cast<int64_t>(r) * IN + c];
    red[threadIdx.x] = sacc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double mean = red[0] / rows;
    __syncthreads();
    double vacc = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const double d = F[static_cast<int64_t>(r) * IN + c] - mean;
        vacc += d * d;
    }
    red[threadIdx.x] = vacc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        params[OFF_MEAN + c] = static_cast<float>(mean);
        params[OFF_SCALE + c] = static_cast<float>(1.0 / fmax(sqrt(red[0] / rows), 1e-6));
    }
}

// Eq. 1 with alpha clamped at -1.999 (finite for binary-like directions).
__device__ __forceinline__ float upsilon_clamped(float a) {
    a = fmaxf(a, -1.999f);
    return a - 2.f * logf(0.5f * a + 1.f);
}

// Raw features of restart r: alpha and step distance of the first kTrajLen iterations, n, log T,
// and Upsilon(alpha at iteration kTrajLen) minus ref (the best among the restarts running then).
__device__ __forceinline__ void restart_features(const float* __restrict__ traj, int r, float n, float logT,
                                                 float ref, float* x) {
#pragma unroll
    for (int t = 0; t < kTrajLen; ++t) {
        x[t] = traj[(static_cast<int64_t>(r) * kTrajLen + t) * 2 + 0];
        x[kTrajLen + t] = traj[(static_cast<int64_t>(r) * kTrajLen + t) * 2 + 1];
    }
    x[10] = n;
    x[11] = logT;
    x[12] = upsilon_clamped(x[kTrajLen - 1]) - ref;
}

// ref = max Upsilon(alpha at iteration kTrajLen) over the restarts running then: the active list
// (act_idx / count) inside a fit, or the restarts with iters[r] >= kTrajLen when recording.
__global__ void upsilon_ref_kernel(const float* __restrict__ traj, const int* __restrict__ act_idx,
                                   const int* __restrict__ count_dev, int count_host, const int* __restrict__ iters,
                                   float* __restrict__ ref) {
    __shared__ float red[256];
    const int count = count_dev ? *count_dev : count_host;
    float m = -INFINITY;
    for (int j = threadIdx.x; j < count; j += blockDim.x) {
        const int r = act_idx ? act_idx[j] : j;
        if (iters && iters[r] < kTrajLen) continue;
        m = fmaxf(m, upsilon_clamped(traj[(static_cast<int64_t>(r) * kTrajLen + kTrajLen - 1) * 2]));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *ref = isfinite(red[0]) ? red[0] : 0.f;
}

// Inference on the active restarts inside a fit: keep flag (p >= tau) per active slot j, and
// the pruned mark of every restart it drops.
__global__ void __launch_bounds__(128) prune_kernel(const float* __restrict__ params, const float* __restrict__ traj,
                                                    const int* __restrict__ act_idx, const int* __restrict__ count_dev,
                                                    int count_host, float n, float logT,
                                                    const float* __restrict__ ref, float tau, float gauss_thr,
                                                    int* __restrict__ keep, int* __restrict__ pruned) {
    __shared__ SmemNet s;
    load_net<true>(params, s);
    const int count = count_dev ? *count_dev : count_host;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const int r = act_idx ? act_idx[j] : j;
    float x[IN];
    restart_features(traj, r, n, logT, *ref, x);
    const float p = sigmoidf(forward_one<true>(s, x, nullptr, nullptr));
    // Gaussian regime: no running restart reaches the Gaussianity threshold (Eq. 3), so no
    // direction of this component is unique; the network keeps nothing (the keep floor decides)
    const bool gaussian = *ref < gauss_thr;
    const int k = (p >= tau && !gaussian) ? 1 : 0;
    keep[j] = k;
    if (!k) pruned[r] = 1;
}

// Keep floor of the pruner: the active restarts with the largest Upsilon(alpha at iteration
// kTrajLen) are kept whatever the network predicts, at least `k` of them: all with Upsilon at or
// above the largest threshold theta that at least k reach (found by bisection over [min, max];
// ties at theta are all kept). The restart leading the objective at that iteration ends at the
// component's pick in most components, so the floor keeps the likely winners; the network adds
// the slower starters. One block.
__global__ void __launch_bounds__(256) keep_top_kernel(const float* __restrict__ traj, const int* __restrict__ act_idx,
                                                       const int* __restrict__ count_dev, int count_host, int k_min,
                                                       float frac, int* __restrict__ keep, int* __restrict__ pruned) {
    __shared__ float rlo[256], rhi[256];
    __shared__ int rc[256];
    const int count = count_dev ? *count_dev : count_host;
    const int tid = threadIdx.x;
    int k = static_cast<int>(ceilf(frac * static_cast<float>(count)));
    if (k < k_min) k = k_min;
    if (k > count) k = count;
    if (k <= 0) return;
    auto u5_of = [&](int j) {
        const int r = act_idx ? act_idx[j] : j;
        return upsilon_clamped(traj[(static_cast<int64_t>(r) * kTrajLen + kTrajLen - 1) * 2]);
    };
    float lo = INFINITY, hi = -INFINITY;
    for (int j = tid; j < count; j += 256) {
        const float u = u5_of(j);
        if (u == u) {  // not NaN
            lo = fminf(lo, u);
            hi = fmaxf(hi, u);
        }
    }
    rlo[tid] = lo;
    rhi[tid] = hi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) {
            rlo[tid] = fminf(rlo[tid], rlo[tid + o]);
            rhi[tid] = fmaxf(rhi[tid], rhi[tid + o]);
        }
        __syncthreads();
    }
    lo = rlo[0];
    hi = rhi[0];
    __syncthreads();
    if (!(lo <= hi)) return;  // every value NaN: the network's decisions stand
    // invariant: count(u >= lo) >= k; find the largest such threshold to FP32 resolution
    float theta = lo;
    for (int it = 0; it < 40 && hi > theta; ++it) {
        const float mid = theta + 0.5f * (hi - theta);
        if (!(mid > theta) || !(mid < hi)) break;
        int c = 0;
        for (int j = tid; j < count; j += 256) c += u5_of(j) >= mid;
        rc[tid] = c;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (tid < o) rc[tid] += rc[tid + o];
            __syncthreads();
        }
        if (rc[0] >= k)
            theta = mid;
        else
            hi = mid;
        __syncthreads();
    }
    {   // hi may itself be reached by k values (a tie at the top): take it when it is
        int c = 0;
        for (int j = tid; j < count; j += 256) c += u5_of(j) >= hi;
        rc[tid] = c;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (tid < o) rc[tid] += rc[tid + o];
            __syncthreads();
        }
        if (rc[0] >= k) theta = hi;
    }
    for (int j = tid; j < count; j += 256)
        if (u5_of(j) >= theta) {
            keep[j] = 1;
            pruned[act_idx ? act_idx[j] : j] = 0;
        }
}

// Redundant restarts: active slot j is dominated when another active restart that leads it in
// Upsilon(alpha at iteration kTrajLen) (larger, or equal with a lower slot) points the same way,
// |b_j . b_j'| >= cos_min (rows are unit vectors after each update). Distinct optima of the
// objective are far apart (the sources' unmixing directions are orthogonal in the whitened space),
// so a dominated restart is heading where a better-placed one already goes; the leader of every
// such cluster is never dominated. Block: 32 slots j against all slots j' in tiles of 32, rows in
// shared memory (stride n_pad + 1: conflict-free); stops scanning once all 32 are dominated.
// Dominated slots leave the keep set (keep[j] = 0, pruned[r] = 1).
constexpr int kDomTile = 32;
__global__ void __launch_bounds__(256) dominated_kernel(const float* __restrict__ B32, int ldb, int n,
                                                        const float* __restrict__ traj,
                                                        const int* __restrict__ act_idx,
                                                        const int* __restrict__ count_dev, int count_host,
                                                        float cos_min, int* __restrict__ keep,
                                                        int* __restrict__ pruned) {
    extern __shared__ float dsm[];
    const int count = count_dev ? *count_dev : count_host;
    const int j0 = blockIdx.x * kDomTile;
    if (j0 >= count) return;
    const int stride = n + 1;
    float* A = dsm;                          // [32][n + 1] rows of this block's slots
    float* Bt = dsm + kDomTile * stride;     // [32][n + 1] rows of the scanned tile
    float* uA = Bt + kDomTile * stride;      // [32] Upsilon of the block's slots
    float* uB = uA + kDomTile;               // [32] Upsilon of the scanned slots
    int* dom = reinterpret_cast<int*>(uB + kDomTile);  // [32]
    __shared__ int all_dom;
    const int tid = threadIdx.x;
    auto row_of = [&](int j) { return act_idx ? act_idx[j] : j; };
    auto u5 = [&](int r) { return upsilon_clamped(traj[(static_cast<int64_t>(r) * kTrajLen + kTrajLen - 1) * 2]); };
    for (int e = tid; e < kDomTile * n; e += 256) {
        const int jj = e / n, k = e % n, j = j0 + jj;
        A[jj * stride + k] = j < count ? B32[static_cast<int64_t>(row_of(j)) * ldb + k] : 0.f;
    }
    if (tid < kDomTile) {
        const int j = j0 + tid;
        uA[tid] = j < count ? u5(row_of(j)) : -INFINITY;
        dom[tid] = j < count ? 0 : 1;
    }
    // thread: slot jj = tid / 8 of the block, scanned slots (tid % 8) * 4 .. + 3
    const int jj = tid >> 3, q0 = (tid & 7) * 4;
    for (int t0 = 0; t0 < count; t0 += kDomTile) {
        __syncthreads();
        if (tid == 0) {
            int a = 1;
            for (int i = 0; i < kDomTile; ++i) a &= dom[i];
            all_dom = a;
        }
        for (int e = tid; e < kDomTile * n; e += 256) {
            const int ii = e / n, k = e % n, j = t0 + ii;
            Bt[ii * stride + k] = j < count ? B32[static_cast<int64_t>(row_of(j)) * ldb + k] : 0.f;
        }
        if (tid < kDomTile) {
            const int j = t0 + tid;
            uB[tid] = j < count ? u5(row_of(j)) : -INFINITY;
        }
        __syncthreads();
        if (all_dom) break;
        const int j = j0 + jj;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < n; ++k) {
            const float a = A[jj * stride + k];
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = fmaf(a, Bt[(q0 + q) * stride + k], d[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jp = t0 + q0 + q;
            if (j < count && jp < count && jp != j) {
                const bool leads = uB[q0 + q] > uA[jj] || (uB[q0 + q] == uA[jj] && jp < j);
                if (leads && fabsf(d[q]) >= cos_min) dom[jj] = 1;  // benign race: every writer stores 1
            }
        }
    }
    __syncthreads();
    if (tid < kDomTile) {
        const int j = j0 + tid;
        if (j < count && dom[tid]) {
            keep[j] = 0;
            pruned[row_of(j)] = 1;
        }
    }
}

// The same test in leading order: the active slots sorted by Upsilon(alpha at iteration kTrajLen),
// descending (ties to the lower slot), by one block (bitonic sort of 64-bit keys in shared
// memory, count <= kDomSortMax). Block b then takes the sorted positions 32 b .. 32 b + 31 and
// scans only the positions before them, tile by tile from the top, stopping once all 32 are
// dominated: a dominated restart usually meets its leader early, and no pair is tested twice.
constexpr int kDomSortMax = 16384;
__device__ __forceinline__ uint32_t desc_key(float u) {
    // order-preserving map of u to an unsigned key, complemented so that larger u sort first;
    // NaN sorts last
    if (u != u) return 0xffffffffu;
    const uint32_t b = __float_as_uint(u);
    const uint32_t asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ~asc;
}
__global__ void __launch_bounds__(1024) lead_sort_kernel(const float* __restrict__ traj, const int* __restrict__ act_idx,
                                                         const int* __restrict__ count_dev, int count_host,
                                                         int* __restrict__ order) {
    extern __shared__ unsigned long long keys[];
    const int count = count_dev ? *count_dev : count_host;
    if (count > kDomSortMax) return;
    int P = 1;
    while (P < count) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < count) {
            const int r = act_idx ? act_idx[i] : i;
            const float u = upsilon_clamped(traj[(static_cast<int64_t>(r) * kTrajLen + kTrajLen - 1) * 2]);
            keys[i] = (static_cast<unsigned long long>(desc_key(u)) << 32) | static_cast<uint32_t>(i);
        } else {
            keys[i] = ~0ull;
        }
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int jb = k >> 1; jb > 0; jb >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int l = i ^ jb;
                if (l > i) {
                    const unsigned long long a = keys[i], b = keys[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < count; i += blockDim.x) order[i] = static_cast<int>(keys[i] & 0xffffffffu);
}
constexpr int kDomSortTile = 64, kDomStride = kDomSortTile + 4;  // k-major tiles, 16-byte aligned rows
__global__ void __launch_bounds__(256) dominated_sorted_kernel(const float* __restrict__ B32, int ldb, int n,
                                                               const int* __restrict__ order,
                                                               const int* __restrict__ act_idx,
                                                               const int* __restrict__ count_dev, int count_host,
                                                               float cos_min, int* __restrict__ keep,
                                                               int* __restrict__ pruned) {
    extern __shared__ __align__(16) float dsm[];
    const int count = count_dev ? *count_dev : count_host;
    const int p0 = blockIdx.x * kDomSortTile;
    if (p0 >= count || count > kDomSortMax) return;
    float* At = dsm;                         // [n][kDomStride]: the block's 64 rows, k-major
    float* Bt = dsm + n * kDomStride;        // [n][kDomStride]: the scanned 64 rows
    __shared__ int dom[kDomSortTile];
    __shared__ int all_dom;
    const int tid = threadIdx.x;
    auto row_at = [&](int pos) {
        const int j = order[pos];
        return act_idx ? act_idx[j] : j;
    };
    for (int e = tid; e < kDomSortTile * n; e += 256) {
        const int rr = e / n, k = e % n, pos = p0 + rr;
        At[k * kDomStride + rr] = pos < count ? B32[static_cast<int64_t>(row_at(pos)) * ldb + k] : 0.f;
    }
    if (tid < kDomSortTile) dom[tid] = p0 + tid < count ? 0 : 1;
    // thread: rows 4 ty .. 4 ty + 3 of the block against scanned rows 4 tx .. 4 tx + 3
    const int ty = tid >> 4, tx = tid & 15;
    for (int t0 = 0; t0 <= p0; t0 += kDomSortTile) {  // positions before the block's, and its own tile
        __syncthreads();
        if (tid == 0) {
            int a = 1;
            for (int i = 0; i < kDomSortTile; ++i) a &= dom[i];
            all_dom = a;
        }
        for (int e = tid; e < kDomSortTile * n; e += 256) {
            const int rr = e / n, k = e % n, pos = t0 + rr;
            Bt[k * kDomStride + rr] = pos < count ? B32[static_cast<int64_t>(row_at(pos)) * ldb + k] : 0.f;
        }
        __syncthreads();
        if (all_dom) break;
        float acc[4][4] = {};
        for (int k = 0; k < n; ++k) {
            const float4 av = *reinterpret_cast<const float4*>(At + k * kDomStride + 4 * ty);
            const float4 bv = *reinterpret_cast<const float4*>(Bt + k * kDomStride + 4 * tx);
            const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a4[i], b4[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int pos = p0 + 4 * ty + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int pp = t0 + 4 * tx + j;  // leads pos when it comes first in the order
                if (pos < count && pp < pos && fabsf(acc[i][j]) >= cos_min) dom[4 * ty + i] = 1;
            }
        }
    }
    __syncthreads();
    if (tid < kDomSortTile) {
        const int pos = p0 + tid;
        if (pos < count && dom[tid]) {
            const int j = order[pos];
            keep[j] = 0;
            pruned[act_idx ? act_idx[j] : j] = 1;
        }
    }
}

// Training record of one component: raw features of every restart and whether the restart
// ended at the picked direction (|b_r . b_p| >= 1 - 1e-3 on normalised rows).
__global__ void record_kernel(const float* __restrict__ traj, const float* __restrict__ B32, int ldb, int n_dim, int M,
                              const int* __restrict__ slot, float n, float logT, const float* __restrict__ ref,
                              float* __restrict__ F_out, float* __restrict__ y_out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    float x[IN];
    restart_features(traj, r, n, logT, *ref, x);
#pragma unroll
    for (int i = 0; i < IN; ++i) F_out[static_cast<int64_t>(r) * IN + i] = x[i];
    const int p = *slot;
    float dot = 0.f, nr = 0.f, np = 0.f;
    for (int k = 0; k < n_dim; ++k) {
        const float a = B32[static_cast<int64_t>(r) * ldb + k], b = B32[static_cast<int64_t>(p) * ldb + k];
        dot = fmaf(a, b, dot);
        nr = fmaf(a, a, nr);
        np = fmaf(b, b, np);
    }
    y_out[r] = fabsf(dot) >= (1.f - 1e-3f) * sqrtf(nr * np) ? 1.f : 0.f;
}

// Fallback test of a pruned component: 1 when some pruned restart's objective when it was pruned
// (Upsilon at iteration kTrajLen, Eq. 1 with alpha clamped at -1.999) is at least the best final
// objective of the restarts that stayed (the pruner may have dropped the global optimum). The
// kurtosis pass covers only the restarts that stayed, so ups holds nothing for the pruned ones.
__global__ void prune_check_kernel(const double* __restrict__ ups, const int* __restrict__ pruned,
                                   const float* __restrict__ traj, int M, int* __restrict__ out) {
    __shared__ double bp[256], bk[256];
    double mp = -INFINITY, mk = -INFINITY;
    for (int r = threadIdx.x; r < M; r += blockDim.x) {
        if (pruned[r])
            mp = fmax(mp, static_cast<double>(
                              upsilon_clamped(traj[(static_cast<int64_t>(r) * kTrajLen + kTrajLen - 1) * 2])));
        else
            mk = fmax(mk, ups[r]);
    }
    bp[threadIdx.x] = mp;
    bk[threadIdx.x] = mk;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            bp[threadIdx.x] = fmax(bp[threadIdx.x], bp[threadIdx.x + o]);
            bk[threadIdx.x] = fmax(bk[threadIdx.x], bk[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = bp[0] >= bk[0] ? 1 : 0;
}
}  // namespace

size_t mlp_scratch_bytes(int rows) {
    const int slices = mlp_slices(rows);
    return sizeof(float) * (static_cast<size_t>(rows) * kActRow + static_cast<size_t>(slices) * kMlpParams +
                            static_cast<size_t>((rows + 127) / 128) + 64);
}

int mlp_slices(int rows) {
    int s = (rows + 511) / 512;
    return s < 1 ? 1 : (s > 32 ? 32 : s);
}

cudaError_t launch_mlp_init(cudaStream_t s, uint64_t seed, float* params) {
    mlp_init_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(seed, params);
    return cudaGetLastError();
}

cudaError_t launch_mlp_standardize(cudaStream_t s, const float* F, int rows, float* params) {
    mlp_standardize_kernel<<<IN, 256, 0, s>>>(F, rows, params);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(cudaStream_t s, const float* params, const float* F, int rows, bool fp16, float* prob) {
    const int blocks = (rows + 127) / 128;
    if (fp16)
        mlp_forward_kernel<true><<<blocks, 128, 0, s>>>(params, F, rows, prob);
    else
        mlp_forward_kernel<false><<<blocks, 128, 0, s>>>(params, F, rows, prob);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train_step(cudaStream_t s, float* params, float* m, float* v, int step, const float* F,
                                  const float* y, int rows, float lr, float pos_weight, bool fp16, float* scratch,
                                  float* loss_out, float* grad_out) {
    const int blocks = (rows + 127) / 128;
    const int slices = mlp_slices(rows);
    const int slice = (rows + slices - 1) / slices;
    float* act = scratch;
    float* gpart = act + static_cast<size_t>(rows) * kActRow;
    float* loss_part = gpart + static_cast<size_t>(slices) * kMlpParams;
    if (fp16)
        mlp_train_fwd_kernel<true><<<blocks, 128, 0, s>>>(params, F, y, rows, pos_weight, act, loss_part);
    else
        mlp_train_fwd_kernel<false><<<blocks, 128, 0, s>>>(params, F, y, rows, pos_weight, act, loss_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mlp_grad_kernel<<<dim3((kMlpParams - 2 * IN + 127) / 128, slices), 128, 0, s>>>(act, rows, slice, gpart);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(params, m, v, gpart, slices, step, lr, grad_out, loss_part,
                                                             blocks, rows, loss_out);
    return cudaGetLastError();
}

cudaError_t launch_prune(cudaStream_t s, const float* params, const float* traj, const int* act_idx,
                         const int* count_dev, int count_host, int n, double logT, float tau, float gauss_thr,
                         float* ref, int* keep, int* pruned, int keep_min, float keep_frac, const float* B32, int ldb,
                         int row_n, float cos_min, int* order) {
    upsilon_ref_kernel<<<1, 256, 0, s>>>(traj, act_idx, count_dev, count_host, nullptr, ref);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prune_kernel<<<(count_host + 127) / 128, 128, 0, s>>>(params, traj, act_idx, count_dev, count_host,
                                                          static_cast<float>(n), static_cast<float>(logT), ref, tau,
                                                          gauss_thr, keep, pruned);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (cos_min > 0.f && B32) {
        const size_t smem = sizeof(float) * (2 * kDomTile * static_cast<size_t>(row_n + 1) + 2 * kDomTile) +
                            sizeof(int) * kDomTile;
        e = allow_max_dyn_smem(dominated_kernel);
        if (e != cudaSuccess) return e;
        if (count_host <= kDomSortMax && order) {
            // count_host bounds the device count: the sorted form runs whenever it is in range
            int P = 1;
            while (P < count_host) P <<= 1;
            e = allow_max_dyn_smem(lead_sort_kernel);
            if (e != cudaSuccess) return e;
            lead_sort_kernel<<<1, 1024, sizeof(unsigned long long) * P, s>>>(traj, act_idx, count_dev, count_host,
                                                                              order);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            e = allow_max_dyn_smem(dominated_sorted_kernel);
            if (e != cudaSuccess) return e;
            const size_t smem_sorted = sizeof(float) * 2 * static_cast<size_t>(row_n) * kDomStride;
            dominated_sorted_kernel<<<(count_host + kDomSortTile - 1) / kDomSortTile, 256, smem_sorted, s>>>(
                B32, ldb, row_n, order, act_idx, count_dev, count_host, cos_min, keep, pruned);
        } else {
            dominated_kernel<<<(count_host + kDomTile - 1) / kDomTile, 256, smem, s>>>(
                B32, ldb, row_n, traj, act_idx, count_dev, count_host, cos_min, keep, pruned);
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess || (keep_min <= 0 && !(keep_frac > 0.f))) return e;
    keep_top_kernel<<<1, 256, 0, s>>>(traj, act_idx, count_dev, count_host, keep_min, keep_frac, keep, pruned);
    return cudaGetLastError();
}

cudaError_t launch_record(cudaStream_t s, const float* traj, const int* iters, const float* B32, int ldb, int n, int M,
                          const int* slot, double logT, float* ref, float* F_out, float* y_out) {
    upsilon_ref_kernel<<<1, 256, 0, s>>>(traj, nullptr, nullptr, M, iters, ref);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    record_kernel<<<(M + 127) / 128, 128, 0, s>>>(traj, B32, ldb, n, M, slot, static_cast<float>(n),
                                                  static_cast<float>(logT), ref, F_out, y_out);
    return cudaGetLastError();
}

cudaError_t launch_prune_check(cudaStream_t s, const double* ups, const int* pruned, const float* traj, int M,
                               int* out) {
    prune_check_kernel<<<1, 256, 0, s>>>(ups, pruned, traj, M, out);
    return cudaGetLastError();
}

}  // namespace ica
