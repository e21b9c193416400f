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
                S.idx[k] = side.indices[lo + c0 + k];
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

// Residual of one refinement step for rows listed in `rows` (their augmented
// systems sit in G_aug, list order): res_a = sum_k w_ka x_ka (r_k -
// sum_c w'_kc x_kc u_c) - reg u_a, with u the current solution, from the FP32
// data and the stored masks (FP32 products, per-thread FP32 sums, FP64
// reduction across the CTA). The residual replaces the rhs column so that a
// second solve of the same G gives the correction.
constexpr int kRefineThreads = 256;

template <int F>
__global__ void __launch_bounds__(kRefineThreads) k_refine_resid(Side side, Params p,
                                                                 const uint32_t* __restrict__ masks,
                                                                 const int32_t* __restrict__ rows, int n_list,
                                                                 float* __restrict__ G_aug,
                                                                 const float* __restrict__ X) {
    constexpr int W = (F + 31) / 32;
    constexpr int PER = (F + 31) / 32;  // columns per lane
    __shared__ double red[kRefineThreads / 32][F];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w = blockIdx.x;
    if (w >= n_list) return;
    const int f = p.f;
    const bool sym = p.gram_mode == GRAM_SYM;
    const int64_t i = rows[w];
    const int64_t lo = side.indptr[i];
    const int n = (int)(side.indptr[i + 1] - lo);
    float u[PER], acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int a = lane + 32 * q;
        u[q] = (a < f) ? X[i * f + a] : 0.f;
        acc[q] = 0.f;
    }
    for (int k = warp; k < n; k += kRefineThreads / 32) {
        const int32_t j = side.indices[lo + k];
        float xv[PER];
        uint32_t mw[W];
#pragma unroll
        for (int q = 0; q < W; ++q) mw[q] = masks[(lo + k) * W + q];
        float dot = 0.f;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int a = lane + 32 * q;
            xv[q] = (a < f) ? __ldg(side.Y + (int64_t)j * f + a) : 0.f;
            const bool wk = (mw[q] >> lane) & 1u;
            if (!sym || wk) dot = fmaf(xv[q], u[q], dot);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) dot += __shfl_xor_sync(kFull, dot, o);
        const float e = side.values[lo + k] - dot;
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if ((mw[q] >> lane) & 1u) acc[q] = fmaf(xv[q], e, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < PER; ++q)
        if (lane + 32 * q < F) red[warp][lane + 32 * q] = (double)acc[q];
    __syncthreads();
    const double reg = p.reg_mode == REG_PLAIN ? (double)p.lambda : (double)p.lambda * (double)n;
    float* aug = G_aug + (int64_t)w * F * (F + 1);
    for (int a = tid; a < F; a += kRefineThreads) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < kRefineThreads / 32; ++q) s += red[q][a];
        const double ua = (a < f) ? (double)X[i * f + a] : 0.0;
        aug[a * (F + 1) + F] = (a < f) ? (float)(s - reg * ua) : 0.f;
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
