// FP64 redo of flagged rows. The FP32 (or mixed-precision) solve appends
// every row whose pivot ratio exceeded the threshold, or whose elimination
// met a zero pivot, to a device list. This kernel re-assembles those rows'
// systems of Eq. core_ui in FP64 from the FP32 data and the stored CES masks
// (products of FP32 values are exact in FP64), adds lambda n_i in FP64, and
// solves by FP64 elimination with partial pivoting (diagonal pivots for the
// symmetric modes). A fixed grid walks the list, whose length it reads on the
// device, so the redo needs no host synchronisation.
#pragma once

#include "als_kernels.cuh"

namespace als {

constexpr int kFp64Threads = 256;
constexpr int kFp64Chunk = 64;

template <int F>
struct Fp64Smem {
    static constexpr int W = (F + 31) / 32;
    double G[F][F + 1];
    double xs[F];
    float x[kFp64Chunk][F];
    float r[kFp64Chunk];
    int32_t idx[kFp64Chunk];
    uint32_t mask[kFp64Chunk][W];
    int piv;
};

template <int F>
__global__ void __launch_bounds__(kFp64Threads) k_fp64_rows(Side side, Params p, const uint32_t* __restrict__ masks,
                                                            const int32_t* __restrict__ list,
                                                            const unsigned int* __restrict__ count,
                                                            float* __restrict__ X_out, int32_t* __restrict__ flags_out,
                                                            Counters* cnt) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using Smem = Fp64Smem<F>;
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    constexpr int W = Smem::W;
    const int tid = threadIdx.x;
    const int f = p.f;
    const bool sym = p.gram_mode == GRAM_SYM;
    const unsigned int total = *count;
    for (unsigned int q = blockIdx.x; q < total; q += gridDim.x) {
        const int64_t i = list[q];
        const int64_t lo = side.indptr[i];
        const int n = (int)(side.indptr[i + 1] - lo);
        for (int e = tid; e < F * (F + 1); e += kFp64Threads) (&S.G[0][0])[e] = 0.0;
        __syncthreads();
        for (int c0 = 0; c0 < n; c0 += kFp64Chunk) {
            const int cn = min(kFp64Chunk, n - c0);
            for (int k = tid; k < cn; k += kFp64Threads) {
                S.idx[k] = factor_row(side.indices[lo + c0 + k], side.n_cols);
                S.r[k] = side.values[lo + c0 + k];
            }
            for (int e = tid; e < cn * W; e += kFp64Threads) (&S.mask[0][0])[e] = masks[(lo + c0) * W + e];
            __syncthreads();
            for (int e = tid; e < cn * F; e += kFp64Threads) {
                const int k = e / F, a = e % F;
                S.x[k][a] = (a < f) ? side.Y[(int64_t)S.idx[k] * f + a] : 0.f;
            }
            __syncthreads();
            // G[a][c] += sum_k w_ka x_ka w'_kc x_kc (c < F), rhs: w_ka x_ka r_k.
            for (int o = tid; o < F * (F + 1); o += kFp64Threads) {
                const int a = o / (F + 1), c = o % (F + 1);
                double acc = 0.0;
                for (int k = 0; k < cn; ++k) {
                    if (!((S.mask[k][a >> 5] >> (a & 31)) & 1u)) continue;
                    double other;
                    if (c == F) {
                        other = (double)S.r[k];
                    } else {
                        if (sym && !((S.mask[k][c >> 5] >> (c & 31)) & 1u)) continue;
                        other = (double)S.x[k][c];
                    }
                    acc = fma((double)S.x[k][a], other, acc);
                }
                S.G[a][c] += acc;
            }
            __syncthreads();
        }
        const double reg = p.reg_mode == REG_PLAIN ? (double)p.lambda : (double)p.lambda * (double)n;
        for (int a = tid; a < F; a += kFp64Threads) S.G[a][a] = (a < f) ? S.G[a][a] + reg : 1.0;
        __syncthreads();
        float ratio;
        const int fl = cta_lu_solve<double, F>(S.G, S.xs, &S.piv, f, p.gram_mode == GRAM_ASYM, p.ratio_max, ratio);
        const bool singular = fl & FLAG_SINGULAR;
        for (int a = tid; a < f; a += kFp64Threads) X_out[i * f + a] = singular ? 0.f : (float)S.xs[a];
        if (tid == 0) {
            if (flags_out) flags_out[i] = fl | FLAG_FP64;
            atomicAdd(&cnt->fp64_rows, 1ull);
        }
        __syncthreads();
    }
}

}  // namespace als

namespace als {

// Residual of one refinement step: res_a = sum_k w_ka x_ka (r_k - sum_c w'_kc
// x_kc u_c) - reg u_a, with u the current solution, from the FP32 data and
// the stored masks (FP32 products and sums, FP64 across chunks of 64
// positions and across lanes). It replaces the rhs column of the row's stored
// system, so that another solve with the same G gives the correction.
// A warp per row (rows of the resident buckets) or a CTA per Gram chunk of a
// split row: G lanes share a position, each holding CPL =
// F / G columns (float4 pieces); the position's dot product x_k . u meets by a
// G-lane shuffle, and each lane keeps FP32 sums of its columns, moved into
// FP64 every 64 positions.
template <int F>
struct ResidCfg {
    static constexpr int W = (F + 31) / 32;
    static constexpr int G = F >= 32 ? 8 : F / 4;  // lanes per position
    static constexpr int CPL = F / G;              // columns per lane (4, 8 or 16)
    static constexpr int PPW = 32 / G;             // positions per warp step
    static_assert(CPL % 4 == 0 && (32 % CPL) == 0, "a lane's columns sit in one mask word, in float4 pieces");
};

// Positions [k0, k1) of the row starting at entry lo into this lane's accd
// (no reduction across the lanes of a column yet).
template <int F>
__device__ __forceinline__ void resid_range(const Side& side, const Params& p, const uint32_t* __restrict__ masks,
                                            int64_t lo, int k0, int k1, const float (&u)[ResidCfg<F>::CPL],
                                            double (&accd)[ResidCfg<F>::CPL]) {
    using R = ResidCfg<F>;
    constexpr int CPL = R::CPL;
    const int lane = threadIdx.x & 31;
    const int g = lane / R::G, c0 = (lane % R::G) * CPL;
    const int f = p.f;
    const bool sym = p.gram_mode == GRAM_SYM;
    const bool vec = f == F && (reinterpret_cast<uintptr_t>(side.Y) & 15u) == 0;
    float acc[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) acc[c] = 0.f;
    for (int kb = k0, it = 0; kb < k1; kb += R::PPW, ++it) {
        const int k = kb + g;
        const bool valid = k < k1;
        float x[CPL];
        uint32_t keep = 0u;
        float rk = 0.f;
        if (valid) {
            const int32_t j = factor_row(side.indices[lo + k], side.n_cols);
            rk = side.values[lo + k];
            keep = masks[(lo + k) * R::W + (c0 >> 5)] >> (c0 & 31);
            if (vec) {
#pragma unroll
                for (int c = 0; c < CPL; c += 4) {
                    const float4 v = __ldg(reinterpret_cast<const float4*>(side.Y + (int64_t)j * F + c0 + c));
                    x[c] = v.x;
                    x[c + 1] = v.y;
                    x[c + 2] = v.z;
                    x[c + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int c = 0; c < CPL; ++c) x[c] = (c0 + c < f) ? __ldg(side.Y + (int64_t)j * f + c0 + c) : 0.f;
            }
        } else {
#pragma unroll
            for (int c = 0; c < CPL; ++c) x[c] = 0.f;
        }
        float dot = 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c)
            if (!sym || ((keep >> c) & 1u)) dot = fmaf(x[c], u[c], dot);
#pragma unroll
        for (int o = 1; o < R::G; o <<= 1) dot += __shfl_xor_sync(kFull, dot, o);
        const float e = rk - dot;
#pragma unroll
        for (int c = 0; c < CPL; ++c)
            if ((keep >> c) & 1u) acc[c] = fmaf(x[c], e, acc[c]);
        if ((it & 63) == 63) {
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                accd[c] += (double)acc[c];
                acc[c] = 0.f;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) accd[c] += (double)acc[c];
}

// This lane's slice of the current solution of row i.
template <int F>
__device__ __forceinline__ void resid_u(const float* __restrict__ X, int64_t i, int f, float (&u)[ResidCfg<F>::CPL]) {
    const int c0 = ((threadIdx.x & 31) % ResidCfg<F>::G) * ResidCfg<F>::CPL;
#pragma unroll
    for (int c = 0; c < ResidCfg<F>::CPL; ++c) u[c] = (c0 + c < f) ? X[i * f + c0 + c] : 0.f;
}

template <int F>
__global__ void __launch_bounds__(256) k_refine_resid_warp(Side side, Params p, const uint32_t* __restrict__ masks,
                                                           const int32_t* __restrict__ rows, int n_list,
                                                           float* __restrict__ G_aug, const float* __restrict__ X) {
    using R = ResidCfg<F>;
    constexpr int CPL = R::CPL;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * 8 + warp;
    if (w >= n_list) return;
    const int64_t i = rows[w];
    const int64_t lo = side.indptr[i];
    const int n = (int)(side.indptr[i + 1] - lo);
    float u[CPL];
    double accd[CPL];
    resid_u<F>(X, i, p.f, u);
#pragma unroll
    for (int c = 0; c < CPL; ++c) accd[c] = 0.0;
    resid_range<F>(side, p, masks, lo, 0, n, u, accd);
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int o = R::G; o < 32; o <<= 1) accd[c] += __shfl_xor_sync(kFull, accd[c], o);
    if (lane < R::G) {
        const double reg = p.reg_mode == REG_PLAIN ? (double)p.lambda : (double)p.lambda * (double)n;
        float* aug = G_aug + (int64_t)w * F * (F + 1);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int a = lane * CPL + c;
            aug[a * (F + 1) + F] = (a < p.f) ? (float)(accd[c] - reg * (double)u[c]) : 0.f;
        }
    }
}

// Split rows: one CTA per Gram chunk writes the chunk's residual partial
// (FP64, F values) to part[c]; k_refine_resid_reduce sums a row's partials
// in chunk order.
template <int F>
__global__ void __launch_bounds__(256) k_refine_resid_chunk(Side side, Params p, SplitPlan sp,
                                                            const uint32_t* __restrict__ masks,
                                                            double* __restrict__ part, const float* __restrict__ X) {
    using R = ResidCfg<F>;
    constexpr int CPL = R::CPL;
    __shared__ double red[8][F];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x;
    const int slot = sp.ch_slot[c];
    const int64_t i = sp.row[slot];
    const int64_t lo = side.indptr[i];
    const int n = (int)(side.indptr[i + 1] - lo);
    const int start = sp.ch_start[c];
    const int len = min(SplitChunk<F>::value, n - start);
    const int per = (len + 7) / 8;
    float u[CPL];
    double accd[CPL];
    resid_u<F>(X, i, p.f, u);
#pragma unroll
    for (int q = 0; q < CPL; ++q) accd[q] = 0.0;
    resid_range<F>(side, p, masks, lo, start + min(warp * per, len), start + min((warp + 1) * per, len), u, accd);
#pragma unroll
    for (int q = 0; q < CPL; ++q)
#pragma unroll
        for (int o = R::G; o < 32; o <<= 1) accd[q] += __shfl_xor_sync(kFull, accd[q], o);
    if (lane < R::G)
#pragma unroll
        for (int q = 0; q < CPL; ++q) red[warp][lane * CPL + q] = accd[q];
    __syncthreads();
    for (int a = threadIdx.x; a < F; a += 256) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) v += red[q][a];
        part[(int64_t)c * F + a] = v;
    }
}

template <int F>
__global__ void k_refine_resid_reduce(Side side, Params p, SplitPlan sp, const double* __restrict__ part,
                                      float* __restrict__ G_aug, const float* __restrict__ X) {
    const int slot = blockIdx.x;
    const int64_t i = sp.row[slot];
    const long long n = side.indptr[i + 1] - side.indptr[i];
    const double reg = p.reg_mode == REG_PLAIN ? (double)p.lambda : (double)p.lambda * (double)n;
    const int c0 = sp.c_begin[slot], c1 = sp.c_begin[slot + 1];
    float* aug = G_aug + (int64_t)slot * F * (F + 1);
    for (int a = threadIdx.x; a < F; a += blockDim.x) {
        double v = 0.0;
        for (int c = c0; c < c1; ++c) v += part[(int64_t)c * F + a];
        aug[a * (F + 1) + F] = (a < p.f) ? (float)(v - reg * (double)X[i * p.f + a]) : 0.f;
    }
}

// X[rows[w]] += D[rows[w]] for the listed rows.
__global__ void k_add_rows(const int32_t* __restrict__ rows, int n_list, int f, const float* __restrict__ D,
                           float* __restrict__ X) {
    const int64_t total = (int64_t)n_list * f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = rows[e / f];
        X[r * f + e % f] += D[r * f + e % f];
    }
}

}  // namespace als
