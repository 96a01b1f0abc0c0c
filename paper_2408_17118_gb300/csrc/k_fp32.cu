// Fused FP32 iteration of the matrix form (Section 3.1; Algorithm 2 update) on CUDA cores:
// for a tile of 64 active restarts and a contiguous sample range, Z = B X~ chunk by chunk in
// registers, Z o Z o Z staged in shared memory, and acc += (Z o Z o Z) X~^T kept in
// registers; Z never reaches device memory. Also accumulates sum z^2, sum z^4 (and
// sum (z^2 - 1)^2 in the moments-only variant used for the kurtosis of candidates).
// Outputs are per-split partial sums, reduced in a fixed order by the finalize kernels.
#include "common.cuh"
#include "internal.h"
#include "rowfin.cuh"

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
// Few-row variant for at most R = 4 or 16 restart rows (the FP32 refinement of the distinct
// best candidates of a component, Algorithm 2's pick made on FP32 data). The work per sample is
// 4 R n FLOPs against n FP32 loads, so the kernel is bound by streaming X~ (from L2: the
// refinement iterations of a component re-read the same X~). Per chunk of CS samples:
//   staging: X~ chunk -> shared memory, transposed to sample-major (row stride n_pad + 4, which
//            keeps both the transposing stores and the 16-byte reads free of bank conflicts);
//            the next chunk's loads are issued into registers before this chunk is computed;
//   pass 1:  thread (sample s, k-part h) forms the partial z_r(s) over its quarter of k for
//            all R rows (b broadcast from shared memory), the parts are summed, and z^3 kept;
//   pass 2:  thread (k-quad q, sample group g) accumulates acc[r][4q..4q+3] += z^3_r(t) x~_t
//            over the samples t = g, g + G, ... of the chunk, in registers across all chunks.
// At the end the per-thread accumulators are summed over g in a fixed order (deterministic).
// ------------------------------------------------------------------------------------------
namespace {
__host__ __device__ constexpr int rows_cs(int n_pad) { return n_pad <= 64 ? 128 : (n_pad <= 128 ? 64 : 32); }
}  // namespace

int fp32_rows_tile(int M_act) { return M_act <= 4 ? 4 : 16; }

size_t fp32_rows_smem_bytes(int n_pad, int R) {
    const int CS = rows_cs(n_pad), SX = n_pad + 4;
    const size_t work = static_cast<size_t>(CS) * SX + 256u * R + static_cast<size_t>(CS) * R;
    const size_t red = 1024u * R;
    return sizeof(float) * (static_cast<size_t>(n_pad) * R + (work > red ? work : red) + 24 * R);
}

// One split (a contiguous range of sample chunks) of the few-row update for rows act_idx[0..M_act)
// by a CTA of 256 threads: partial (z o z o z) X~^T (or the moments) of the split into
// part_acc / part_mom. rsm: the CTA's dynamic shared memory (fp32_rows_smem_bytes). Restart
// rows and the list are read with cache-global loads (the persistent refinement rewrites them
// between its updates).
template <int R, bool MOMENTS_ONLY>
__device__ __forceinline__ void rows_update(const float* __restrict__ B32, int ldb, const int* __restrict__ act_idx,
                                            int M_act, const float* __restrict__ Xt, int64_t ldx, int n_pad,
                                            int64_t T, int chunks_per_split, int split, float* __restrict__ part_acc,
                                            float* __restrict__ part_mom, int part_rows, float* rsm) {
    const int CS = rows_cs(n_pad), SX = n_pad + 4, H = 256 / CS, KQ = n_pad / 4, G = 256 / KQ;
    float* Bs = rsm;                    // [n_pad][R]
    float* Xs = Bs + n_pad * R;         // [CS][SX]   sample-major X~ chunk
    float* zp = Xs + CS * SX;           // [H][CS][R] partial z
    float* z3 = zp + 256 * R;           // [CS][R]    z^3
    float* red = Xs;                    // [G][R][n_pad] end-of-kernel reduction (aliases the above)
    const size_t work = static_cast<size_t>(CS) * SX + 256u * R + static_cast<size_t>(CS) * R;
    float* redm = Xs + (work > 1024u * R ? work : 1024u * R);  // [8][R][3]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < n_pad * R; e += 256) {
        const int k = e / R, r = e % R;
        float v = 0.f;
        if (r < M_act) v = __ldcg(B32 + static_cast<int64_t>(act_idx ? __ldcg(act_idx + r) : r) * ldb + k);
        Bs[e] = v;
    }
    const int64_t total_chunks = (T + CS - 1) / CS;
    const int64_t c_begin = static_cast<int64_t>(split) * chunks_per_split;
    const int64_t c_end = c_begin + chunks_per_split < total_chunks ? c_begin + chunks_per_split : total_chunks;

    // staging map: a warp instruction covers 4 consecutive k x 8 consecutive samples
    const int n_el = CS * n_pad;  // <= 8192: at most 32 per thread
    float pre[32];
    auto load_chunk = [&](int64_t c) {
        const int64_t t0 = c * CS;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int e = tid + 256 * j;
            if (e >= n_el) break;
            const int wi = e >> 5, l = e & 31;
            const int k = 4 * (wi % KQ) + (l & 3), t = 8 * (wi / KQ) + (l >> 2);
            pre[j] = (t0 + t < T) ? __ldg(Xt + static_cast<int64_t>(k) * ldx + t0 + t) : 0.f;
        }
    };
    auto store_chunk = [&]() {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int e = tid + 256 * j;
            if (e >= n_el) break;
            const int wi = e >> 5, l = e & 31;
            const int k = 4 * (wi % KQ) + (l & 3), t = 8 * (wi / KQ) + (l >> 2);
            Xs[t * SX + k] = pre[j];
        }
    };

    float acc[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[r][j] = 0.f;
    float m2 = 0.f, m4 = 0.f, mq = 0.f;  // moments of row tid % R
    const int s1 = tid % CS, h1 = tid / CS;
    const int q_lo = h1 * KQ / H, q_hi = (h1 + 1) * KQ / H;
    const int q2 = tid % KQ, g2 = tid / KQ;

    if (c_begin < c_end) load_chunk(c_begin);
    for (int64_t c = c_begin; c < c_end; ++c) {
        const int64_t t0 = c * CS;
        __syncthreads();  // the previous chunk's readers are done with Xs / z3
        store_chunk();
        __syncthreads();
        if (c + 1 < c_end) load_chunk(c + 1);
        // pass 1: partial z over this thread's k-part, all R rows
        {
            float z[R];
#pragma unroll
            for (int r = 0; r < R; ++r) z[r] = 0.f;
            for (int q = q_lo; q < q_hi; ++q) {
                const float4 x = *reinterpret_cast<const float4*>(&Xs[s1 * SX + 4 * q]);
                const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
#pragma unroll
                    for (int r4 = 0; r4 < R; r4 += 4) {
                        const float4 b = *reinterpret_cast<const float4*>(&Bs[(4 * q + j) * R + r4]);
                        z[r4 + 0] = fmaf(b.x, xv[j], z[r4 + 0]);
                        z[r4 + 1] = fmaf(b.y, xv[j], z[r4 + 1]);
                        z[r4 + 2] = fmaf(b.z, xv[j], z[r4 + 2]);
                        z[r4 + 3] = fmaf(b.w, xv[j], z[r4 + 3]);
                    }
                }
            }
#pragma unroll
            for (int r4 = 0; r4 < R; r4 += 4)
                *reinterpret_cast<float4*>(&zp[(h1 * CS + s1) * R + r4]) = make_float4(z[r4], z[r4 + 1], z[r4 + 2], z[r4 + 3]);
        }
        __syncthreads();
        // z = sum of the parts; moments; z^3
        for (int i = tid; i < CS * R; i += 256) {
            const int s = i / R;
            float z = 0.f;
            for (int h = 0; h < H; ++h) z += zp[(h * CS + s) * R + (i % R)];
            const float zz = z * z;
            m2 += zz;
            m4 = fmaf(zz, zz, m4);
            if (MOMENTS_ONLY) {
                const float e = (t0 + s < T) ? zz - 1.f : 0.f;
                mq = fmaf(e, e, mq);
            } else {
                z3[i] = zz * z;
            }
        }
        if (!MOMENTS_ONLY) {
            __syncthreads();
            // pass 2: acc[r][4 q2 + j] += z^3_r(t) x~[t][4 q2 + j]
            if (g2 < G) {
                for (int t = g2; t < CS; t += G) {
                    const float4 x = *reinterpret_cast<const float4*>(&Xs[t * SX + 4 * q2]);
#pragma unroll
                    for (int r4 = 0; r4 < R; r4 += 4) {
                        const float4 zc = *reinterpret_cast<const float4*>(&z3[t * R + r4]);
                        const float zv[4] = {zc.x, zc.y, zc.z, zc.w};
#pragma unroll
                        for (int rr = 0; rr < 4; ++rr) {
                            acc[r4 + rr][0] = fmaf(zv[rr], x.x, acc[r4 + rr][0]);
                            acc[r4 + rr][1] = fmaf(zv[rr], x.y, acc[r4 + rr][1]);
                            acc[r4 + rr][2] = fmaf(zv[rr], x.z, acc[r4 + rr][2]);
                            acc[r4 + rr][3] = fmaf(zv[rr], x.w, acc[r4 + rr][3]);
                        }
                    }
                }
            }
        }
    }
    // moments: threads with the same tid % R hold the same row
#pragma unroll
    for (int o = R; o < 32; o <<= 1) {
        m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        m4 += __shfl_xor_sync(0xffffffffu, m4, o);
        mq += __shfl_xor_sync(0xffffffffu, mq, o);
    }
    __syncthreads();  // every reader of Xs / zp / z3 is done: the reduction area may alias them
    if (lane < R) {
        redm[(warp * R + lane) * 3 + 0] = m2;
        redm[(warp * R + lane) * 3 + 1] = m4;
        redm[(warp * R + lane) * 3 + 2] = mq;
    }
    if (!MOMENTS_ONLY && g2 < G) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            *reinterpret_cast<float4*>(&red[(g2 * R + r) * n_pad + 4 * q2]) =
                make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    }
    __syncthreads();
    if (tid < R && tid < M_act) {
        float a2 = 0.f, a4 = 0.f, aq = 0.f;
        for (int w = 0; w < 8; ++w) {
            a2 += redm[(w * R + tid) * 3 + 0];
            a4 += redm[(w * R + tid) * 3 + 1];
            aq += redm[(w * R + tid) * 3 + 2];
        }
        float* pm = part_mom + (static_cast<int64_t>(split) * part_rows + tid) * 4;
        pm[0] = a2;
        pm[1] = a4;
        pm[2] = aq;
        pm[3] = 0.f;
    }
    if (!MOMENTS_ONLY) {
        for (int o = tid; o < R * n_pad; o += 256) {
            const int r = o / n_pad, k = o % n_pad;
            if (r >= M_act) continue;
            float v = 0.f;
            for (int g = 0; g < G; ++g) v += red[(g * R + r) * n_pad + k];
            part_acc[(static_cast<int64_t>(split) * part_rows + r) * n_pad + k] = v;
        }
    }
}

template <int R, bool MOMENTS_ONLY>
__global__ void __launch_bounds__(256) fused_fp32_rows_kernel(const float* __restrict__ B32, int ldb,
                                                              const int* __restrict__ act_idx,
                                                              const int* __restrict__ count_dev, int M_act_host,
                                                              const float* __restrict__ Xt, int64_t ldx, int n_pad,
                                                              int64_t T, int chunks_per_split,
                                                              float* __restrict__ part_acc,
                                                              float* __restrict__ part_mom, int part_rows) {
    extern __shared__ __align__(16) float rsm[];
    pdl_wait();  // the refinement loop's previous finalize wrote B, the list and the count
    pdl_trigger();
    const int M_act = count_dev ? *count_dev : M_act_host;
    rows_update<R, MOMENTS_ONLY>(B32, ldb, act_idx, M_act, Xt, ldx, n_pad, T, chunks_per_split, blockIdx.x, part_acc,
                                 part_mom, part_rows, rsm);
}

template <int R>
cudaError_t launch_rows_variant(cudaStream_t s, bool moments_only, const float* B32, int ldb, const int* act_idx,
                                const int* count_dev, int M_act_host, const float* Xt, int64_t ldx, int n_pad,
                                int64_t T, int splits, int chunks_per_split, float* part_acc, float* part_mom,
                                int part_rows, bool pdl) {
    const size_t smem = fp32_rows_smem_bytes(n_pad, R);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(splits), 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e;
    if (moments_only) {
        e = allow_max_dyn_smem(fused_fp32_rows_kernel<R, true>);
        if (e != cudaSuccess) return e;
        return cudaLaunchKernelEx(&cfg, fused_fp32_rows_kernel<R, true>, B32, ldb, act_idx, count_dev, M_act_host, Xt,
                                  ldx, n_pad, T, chunks_per_split, part_acc, part_mom, part_rows);
    }
    e = allow_max_dyn_smem(fused_fp32_rows_kernel<R, false>);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, fused_fp32_rows_kernel<R, false>, B32, ldb, act_idx, count_dev, M_act_host, Xt,
                              ldx, n_pad, T, chunks_per_split, part_acc, part_mom, part_rows);
}

int fp32_rows_chunk(int n_pad) { return rows_cs(n_pad); }

cudaError_t launch_fused_fp32_rows(cudaStream_t s, bool moments_only, const float* B32, int ldb, const int* act_idx,
                                   const int* count_dev, int M_act_host, const float* Xt, int64_t ldx, int n_pad,
                                   int64_t T, int splits, int chunks_per_split, float* part_acc, float* part_mom,
                                   int part_rows, bool pdl) {
    if (part_rows == 4)
        return launch_rows_variant<4>(s, moments_only, B32, ldb, act_idx, count_dev, M_act_host, Xt, ldx, n_pad, T,
                                      splits, chunks_per_split, part_acc, part_mom, part_rows, pdl);
    if (part_rows == 16)
        return launch_rows_variant<16>(s, moments_only, B32, ldb, act_idx, count_dev, M_act_host, Xt, ldx, n_pad, T,
                                       splits, chunks_per_split, part_acc, part_mom, part_rows, pdl);
    return cudaErrorInvalidValue;
}

cudaError_t launch_fused_fp32(cudaStream_t s, bool moments_only, const float* B32, int ldb, const int* act_idx,
                              const int* count_dev, int M_act, const float* Xt, int64_t ldx, int n_pad, int64_t T,
                              int splits, int chunks_per_split, float* part_acc, float* part_mom, int part_rows) {
    const size_t smem = fp32_smem_bytes(n_pad);
    const dim3 grid(splits, (M_act + F_MT - 1) / F_MT);
    cudaError_t e;
    if (moments_only) {
        e = allow_max_dyn_smem(fused_fp32_kernel<true>);
        if (e != cudaSuccess) return e;
        fused_fp32_kernel<true><<<grid, 256, smem, s>>>(B32, ldb, act_idx, count_dev, M_act, Xt, ldx, n_pad, T,
                                                        chunks_per_split, part_acc, part_mom, part_rows);
    } else {
        e = allow_max_dyn_smem(fused_fp32_kernel<false>);
        if (e != cudaSuccess) return e;
        fused_fp32_kernel<false><<<grid, 256, smem, s>>>(B32, ldb, act_idx, count_dev, M_act, Xt, ldx, n_pad, T,
                                                         chunks_per_split, part_acc, part_mom, part_rows);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Persistent FP32 refinement (a8): every refinement iteration of the few candidate rows in one
// cooperative launch, one CTA per split of the sample range (the per-launch loop's grid).
// Per iteration: the few-row update of the CTA's split (rows_update); grid barrier; CTA j
// finishes active row j (its 8 warps sum the split partials in the order of finalize_kernel<32>:
// 32 virtual warps, warp w taking virtual warps w, w + 8, ...); grid barrier; every CTA compacts
// the list of rows still moving. Same arithmetic as the per-launch loop (fused_fp32_rows_kernel +
// finalize_kernel<32>), so both give identical rows.
// ------------------------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(256, 2) refine_fp32_kernel(RefineLaunch a, int chunks_per_split) {
    extern __shared__ __align__(16) float rsm[];
    __shared__ int new_count;
    __shared__ int abort_sh;
    volatile int* abort_flag = &abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int G = static_cast<int>(gridDim.x), bid = static_cast<int>(blockIdx.x);
    if (tid == 0) abort_sh = 0;
    __syncthreads();
    const int nq = (a.n_pad + 31) >> 5;
    unsigned int target = 0;
    int cur = a.cur0;
    int M_act = __ldcg(cur ? a.count1 : a.count0);
    int t = a.t_begin;
    for (; t < a.t_end && M_act > 0; ++t) {
        const int* act = cur ? a.act1 : a.act0;
        rows_update<R, false>(a.B32, a.ldb, act, M_act, a.Xt, a.ldx, a.n_pad, a.T, chunks_per_split, bid, a.part_acc,
                              a.part_mom, R, rsm);
        target += static_cast<unsigned int>(G);
        if (!grid_barrier(a.bar_ctr, target, abort_flag, a.status, a.wait_ns ? a.wait_ns : ICA_WAIT_NS)) break;
        if (bid < M_act) {  // row j = bid
            const int j = bid;
            int r = 0;
            float b[8];
            if (warp == 0) {
                r = __ldcg(act + j);
                load_row(a.B32, a.ldb, r, nq, a.n, b);
            }
            row_partials(a.part_acc, a.part_mom, G, R, a.n_pad, j, false, 32, 8, warp, rsm);
            __syncthreads();
            if (warp == 0) {
                float accv[8], e2, e4;
                row_combine(rsm, 32, a.n_pad, a.n, false, accv, &e2, &e4);
                finish_row_loaded(accv, b, nq, a.n, r, j, a.B32, a.ldb, a.inv_T, a.tol, a.flags, a.iters, nullptr,
                                  kTrajLen, false, 0.f, 0.f, a.status, RowProj{a.Wp, a.Wp ? a.nw : 0, a.ldw});
            }
        }
        target += static_cast<unsigned int>(G);
        if (!grid_barrier(a.bar_ctr, target, abort_flag, a.status, a.wait_ns ? a.wait_ns : ICA_WAIT_NS)) break;
        compact_block(a.flags, act, M_act, cur ? a.act0 : a.act1, &new_count, bid == 0 ? a.rows_accum : nullptr, 256);
        __syncthreads();
        const int M_new = *reinterpret_cast<volatile int*>(&new_count);
        __syncthreads();
        cur ^= 1;
        M_act = M_new;
    }
    if (bid == 0 && tid == 0 && !abort_sh) {
        a.ctl[0] = t;
        a.ctl[1] = M_act;
        a.ctl[2] = cur;
        *(cur ? a.count1 : a.count0) = M_act;
    }
}

cudaError_t launch_refine_fp32(cudaStream_t s, const RefineLaunch& p, int* resident) {
    constexpr int R = 4;
    if (p.rows_max > R || p.n_pad > kMaxN) return cudaErrorInvalidValue;
    const int64_t total = (p.T + rows_cs(p.n_pad) - 1) / rows_cs(p.n_pad);
    if (p.splits < 1 || static_cast<int64_t>(p.splits) * p.cps < total) return cudaErrorInvalidValue;
    // the finish step sums 32 virtual warps' partials in the kernel's shared memory
    size_t smem = fp32_rows_smem_bytes(p.n_pad, R);
    const size_t fin = sizeof(float) * 32 * (2 * static_cast<size_t>(p.n_pad) + 4);
    if (fin > smem) smem = fin;
    cudaError_t e = allow_max_dyn_smem(refine_fp32_kernel<R>);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refine_fp32_kernel<R>, 256, smem)) != cudaSuccess)
        return e;
    if (resident) *resident = per_sm * sms;
    if (per_sm * sms < p.splits) return cudaErrorCooperativeLaunchTooLarge;  // nothing launched
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(p.splits), 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, refine_fp32_kernel<R>, p, p.cps);
}

}  // namespace ica
