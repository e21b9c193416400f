// Kernels of one Core-ALS half-sweep on CUDA cores (FP32), n_f <= 32.
//
// Rows are bucketed by length by the host planner:
//   * k_warp_rows : n_i <= 32. One warp per row does CES (Algorithm 1),
//                   the Gram assembly of Eq. (core_ui) and the solve, all in
//                   registers and a warp-private shared-memory tile.
//   * k_cta_rows  : n_i > 32. One CTA per row does CES by an exact radix
//                   select over shared-memory histograms and the masked Gram
//                   assembly; the augmented system [G | b] goes to the
//                   workspace and k_solve_rows solves it (warp per row).
//                   Rows up to kCtaResident elements are staged in shared
//                   memory once; longer rows are streamed from L2 per pass.
#pragma once

#include "als_device.cuh"

namespace als {

constexpr int kWarpRowMax = 32;
constexpr int kCtaThreads = 256;
constexpr int kCtaWarps = kCtaThreads / 32;
constexpr int kCtaResident = 256;

// ---------------------------------------------------------------------------
// Warp per row (n_i <= 32).
// mode 0: solve and write X; 1: write the augmented system to G_aug (indexed
// by list position); 2: masks only.
template <int F>
struct WarpRowTile {
    union {
        float x[32][F + 1];
        float G[F][F + 2];
    } u;
    float r[32];
    int32_t idx[32];
    uint32_t sel[F];
};

template <int F>
__global__ void __launch_bounds__(256) k_warp_rows(Side side, Params p, const int32_t* __restrict__ rows,
                                                   int n_list, int mode, float* __restrict__ X_out,
                                                   int32_t* __restrict__ flags_out,
                                                   uint32_t* __restrict__ masks_out,
                                                   float* __restrict__ G_aug, Counters* cnt) {
    __shared__ WarpRowTile<F> tiles[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * 8 + warp;
    if (w >= n_list) return;
    WarpRowTile<F>& T = tiles[warp];
    const int f = p.f;
    const int64_t i = rows[w];
    const int64_t lo = side.indptr[i];
    const int n = (int)(side.indptr[i + 1] - lo);

    if (lane < n) {
        T.idx[lane] = side.indices[lo + lane];
        T.r[lane] = side.values[lo + lane];
    }
    __syncwarp();
    for (int e = lane; e < n * F; e += 32) {
        const int k = e / F, a = e % F;
        T.u.x[k][a] = (a < f) ? __ldg(side.Y + (int64_t)T.idx[k] * f + a) : 0.f;
    }
    __syncwarp();

    const int s = (int)row_budget(n, p);
    for (int a = 0; a < F; ++a) {
        unsigned m = 0u;
        if (a < f) {
            uint32_t key = (lane < n) ? mag_key(T.u.x[lane][a]) : 0u;
            m = warp_ces_column(key, n, s);
        }
        if (lane == 0) T.sel[a] = m;
    }
    __syncwarp();
    if (masks_out != nullptr && lane < n) {
        uint32_t word = 0u;
        for (int a = 0; a < f; ++a) word |= ((T.sel[a] >> lane) & 1u) << a;
        masks_out[lo + lane] = word;
    }
    if (mode == 2) return;

    // Masked Gram: G[a][b] = sum_k w_ka x_ka w'_kb x_kb, b_a = sum_k w_ka x_ka r_k
    // with w the keep mask and w' = w (symmetric variant) or 1.
    constexpr int TA = F / 8, TB = F / 4;
    const int ta = lane >> 2, tb = lane & 3;
    const int a0 = ta * TA, b0 = tb * TB;
    const bool sym = (p.gram_mode == GRAM_SYM);
    uint32_t sa[TA], sb[TB];
#pragma unroll
    for (int q = 0; q < TA; ++q) sa[q] = T.sel[a0 + q];
#pragma unroll
    for (int q = 0; q < TB; ++q) sb[q] = sym ? T.sel[b0 + q] : kFull;
    float acc[TA][TB];
    float rh[TA];
#pragma unroll
    for (int q = 0; q < TA; ++q) {
        rh[q] = 0.f;
#pragma unroll
        for (int t = 0; t < TB; ++t) acc[q][t] = 0.f;
    }
    for (int k = 0; k < n; ++k) {
        float xa[TA], xb[TB];
#pragma unroll
        for (int q = 0; q < TA; ++q) xa[q] = ((sa[q] >> k) & 1u) ? T.u.x[k][a0 + q] : 0.f;
#pragma unroll
        for (int t = 0; t < TB; ++t) xb[t] = ((sb[t] >> k) & 1u) ? T.u.x[k][b0 + t] : 0.f;
        const float rk = T.r[k];
#pragma unroll
        for (int q = 0; q < TA; ++q) {
            rh[q] = fmaf(xa[q], rk, rh[q]);
#pragma unroll
            for (int t = 0; t < TB; ++t) acc[q][t] = fmaf(xa[q], xb[t], acc[q][t]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < TA; ++q) {
#pragma unroll
        for (int t = 0; t < TB; ++t) T.u.G[a0 + q][b0 + t] = acc[q][t];
        if (tb == 0) T.u.G[a0 + q][F] = rh[q];
    }
    __syncwarp();
    if (lane < F) {
        const float reg = row_reg(n, p);
        T.u.G[lane][lane] = (lane < f) ? T.u.G[lane][lane] + reg : 1.f;
    }
    __syncwarp();
    if (mode == 1) {
        float* dst = G_aug + (int64_t)w * F * (F + 1);
        for (int e = lane; e < F * (F + 1); e += 32) dst[e] = T.u.G[e / (F + 1)][e % (F + 1)];
        return;
    }
    float v[F];
#pragma unroll
    for (int j = 0; j < F; ++j) v[j] = (lane < F) ? T.u.G[lane][j] : 0.f;
    const float rhs = (lane < F) ? T.u.G[lane][F] : 0.f;
    float x;
    int flags;
    float ratio;
    warp_solve<F>(v, rhs, f, p.gram_mode == GRAM_ASYM, p.ratio_max, x, flags, ratio);
    if (lane < f) X_out[i * f + lane] = x;
    if (lane == 0) {
        if (flags_out) flags_out[i] = flags;
        record_flags(cnt, flags, ratio);
    }
}

// ---------------------------------------------------------------------------
// CTA per row (n_i > 32).
template <int F>
struct CtaRowSmem {
    float x[kCtaResident][F];
    float r[kCtaResident];
    int32_t idx[kCtaResident];
    uint32_t mask[kCtaResident];
    union {
        uint32_t hist[F][256];
        float Gp[kCtaWarps][F][F + 1];
    } u;
    uint32_t P[F];     // resolved high-bit prefix of the threshold key
    uint32_t Mk[F];    // bits of the key covered by P
    int32_t need[F];   // elements still to take inside the prefix class
    int32_t cut[F];    // positional cut among keys equal to P (INT_MAX = none)
    int32_t done[F];
    int32_t active;
};

template <int F>
__device__ __forceinline__ void cta_stage(CtaRowSmem<F>& S, const Side& side, int f, int64_t lo, int c0, int cn) {
    for (int k = threadIdx.x; k < cn; k += kCtaThreads) {
        S.idx[k] = side.indices[lo + c0 + k];
        S.r[k] = side.values[lo + c0 + k];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cn * F; e += kCtaThreads) {
        const int k = e / F, a = e % F;
        S.x[k][a] = (a < f) ? __ldg(side.Y + (int64_t)S.idx[k] * f + a) : 0.f;
    }
    __syncthreads();
}

template <int F>
__global__ void __launch_bounds__(kCtaThreads) k_cta_rows(Side side, Params p, const int32_t* __restrict__ rows,
                                                          int n_list, int mode, float* __restrict__ G_aug,
                                                          uint32_t* __restrict__ masks_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaRowSmem<F>& S = *reinterpret_cast<CtaRowSmem<F>*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w = blockIdx.x;
    if (w >= n_list) return;
    const int f = p.f;
    const int64_t i = rows[w];
    const int64_t lo = side.indptr[i];
    const int n = (int)(side.indptr[i + 1] - lo);
    const bool resident = n <= kCtaResident;
    const int s = (int)row_budget(n, p);
    // Thread t always handles column a_t = t mod F (F divides the block size).
    const int a_t = tid % F;
    const int k0 = tid / F;
    constexpr int kstep = kCtaThreads / F;

    if (tid < F) {
        const bool real = tid < f;
        S.need[tid] = s;
        S.cut[tid] = 0x7fffffff;
        if (!real || s == 0) {  // keep nothing
            S.P[tid] = 0xffffffffu;
            S.Mk[tid] = 0xffffffffu;
            S.cut[tid] = 0;
            S.done[tid] = 1;
        } else if (s >= n) {  // keep everything
            S.P[tid] = 0u;
            S.Mk[tid] = 0u;
            S.done[tid] = 1;
        } else {
            S.P[tid] = 0u;
            S.Mk[tid] = 0u;
            S.done[tid] = 0;
        }
    }
    if (tid == 0) S.active = (f > 0 && s > 0 && s < n) ? 1 : 0;
    if (resident) cta_stage<F>(S, side, f, lo, 0, n);
    __syncthreads();

    // ---- Radix select of the s-th largest key, 8 bits per pass, per column.
    for (int pass = 0; pass < 4; ++pass) {
        if (!S.active) break;
        const int shift = 24 - 8 * pass;
        const uint32_t hm = pass == 0 ? 0u : (0xffffffffu << (32 - 8 * pass));
        for (int e = tid; e < F * 256; e += kCtaThreads) (&S.u.hist[0][0])[e] = 0u;
        __syncthreads();
        const bool mine = !S.done[a_t];
        const uint32_t Pa = S.P[a_t];
        for (int c0 = 0; c0 < n; c0 += kCtaResident) {
            const int cn = min(kCtaResident, n - c0);
            if (!resident) cta_stage<F>(S, side, f, lo, c0, cn);
            if (mine) {
                for (int k = k0; k < cn; k += kstep) {
                    const uint32_t key = mag_key(S.x[k][a_t]);
                    if ((key & hm) == Pa) atomicAdd(&S.u.hist[a_t][(key >> shift) & 255u], 1u);
                }
            }
            if (!resident) __syncthreads();
        }
        __syncthreads();
        // Scan: one warp per column, bins from the top.
        for (int a = warp; a < F; a += kCtaWarps) {
            if (S.done[a]) continue;
            uint32_t c[8];
            uint32_t lsum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = S.u.hist[a][lane * 8 + q];
                lsum += c[q];
            }
            uint32_t incl = lsum;  // sum over lanes >= this lane
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_down_sync(kFull, incl, o);
                if (lane + o < 32) incl += t;
            }
            const uint32_t above = incl - lsum;
            const uint32_t nd = (uint32_t)S.need[a];
            const bool owner = above < nd && nd <= incl;
            const unsigned ob = __ballot_sync(kFull, owner);
            const int L = __ffs(ob) - 1;
            int digit = 0;
            uint32_t newneed = 0, inbin = 0;
            if (lane == L) {
                uint32_t cum = above;
#pragma unroll
                for (int q = 7; q >= 0; --q) {
                    if (cum + c[q] >= nd && inbin == 0) {
                        digit = lane * 8 + q;
                        newneed = nd - cum;
                        inbin = c[q];
                    }
                    if (inbin == 0) cum += c[q];
                }
            }
            digit = __shfl_sync(kFull, digit, L);
            newneed = __shfl_sync(kFull, newneed, L);
            inbin = __shfl_sync(kFull, inbin, L);
            if (lane == 0) {
                S.P[a] |= (uint32_t)digit << shift;
                S.Mk[a] = hm | (0xffu << shift);
                S.need[a] = (int)newneed;
                if (inbin == newneed) S.done[a] = 1;  // the whole class is kept
            }
        }
        __syncthreads();
        if (tid == 0) {
            int act = 0;
            for (int a = 0; a < F; ++a) act |= !S.done[a];
            S.active = act;
        }
        __syncthreads();
    }
    // Columns still open have the full threshold key P and more equal keys
    // than places: keep the lowest positions (cut = one past the last kept).
    for (int a = warp; a < F; a += kCtaWarps) {
        if (S.done[a]) continue;
        const uint32_t T = S.P[a];
        const int nd = S.need[a];
        int seen = 0, cut = n;
        for (int kb = 0; kb < n; kb += 32) {
            const int k = kb + lane;
            bool eq = false;
            if (k < n) {
                const float xv = resident ? S.x[k][a]
                                          : __ldg(side.Y + (int64_t)side.indices[lo + k] * f + a);
                eq = mag_key(xv) == T;
            }
            unsigned b = __ballot_sync(kFull, eq);
            const int c = __popc(b);
            if (seen + c >= nd) {
                int want = nd - seen;
                while (--want > 0) b &= b - 1u;
                cut = kb + __ffs(b);  // position of the last kept one, plus one
                break;
            }
            seen += c;
        }
        if (lane == 0) S.cut[a] = cut;
    }
    __syncthreads();

    // ---- Masked Gram over the row, warps split the positions.
    constexpr int TA = F / 8, TB = F / 4;
    const int ta = lane >> 2, tb = lane & 3;
    const int a0 = ta * TA, b0 = tb * TB;
    const bool sym = (p.gram_mode == GRAM_SYM);
    float acc[TA][TB];
    float rh[TA];
#pragma unroll
    for (int q = 0; q < TA; ++q) {
        rh[q] = 0.f;
#pragma unroll
        for (int t = 0; t < TB; ++t) acc[q][t] = 0.f;
    }
    const uint32_t Pa = S.P[a_t], Ma = S.Mk[a_t];
    const int cuta = S.cut[a_t];
    const uint32_t fmask = (F == 32) ? kFull : ((1u << F) - 1u);
    for (int c0 = 0; c0 < n; c0 += kCtaResident) {
        const int cn = min(kCtaResident, n - c0);
        if (!resident) cta_stage<F>(S, side, f, lo, c0, cn);
        // Keep masks of this chunk: thread (k, a_t) decides, a ballot packs.
        for (int kk = 0; kk < cn; kk += kstep) {
            const int k = kk + k0;
            bool keep = false;
            if (k < cn) {
                const uint32_t key = mag_key(S.x[k][a_t]) & Ma;
                keep = key > Pa || (key == Pa && (c0 + k) < cuta);
            }
            const unsigned b = __ballot_sync(kFull, keep);
            if (a_t == 0 && k < cn) S.mask[k] = (b >> (lane & ~(F - 1))) & fmask;
        }
        __syncthreads();
        if (masks_out != nullptr) {
            for (int k = tid; k < cn; k += kCtaThreads) masks_out[lo + c0 + k] = S.mask[k] & ((f == 32) ? kFull : ((1u << f) - 1u));
        }
        if (mode != 2) {
            for (int k = warp; k < cn; k += kCtaWarps) {
                const uint32_t m = S.mask[k];
                float xa[TA], xb[TB];
#pragma unroll
                for (int q = 0; q < TA; ++q) xa[q] = ((m >> (a0 + q)) & 1u) ? S.x[k][a0 + q] : 0.f;
#pragma unroll
                for (int t = 0; t < TB; ++t)
                    xb[t] = (!sym || ((m >> (b0 + t)) & 1u)) ? S.x[k][b0 + t] : 0.f;
                const float rk = S.r[k];
#pragma unroll
                for (int q = 0; q < TA; ++q) {
                    rh[q] = fmaf(xa[q], rk, rh[q]);
#pragma unroll
                    for (int t = 0; t < TB; ++t) acc[q][t] = fmaf(xa[q], xb[t], acc[q][t]);
                }
            }
        }
        __syncthreads();
    }
    if (mode == 2) return;
    // Per-warp partials, then a fixed-order reduction over warps.
#pragma unroll
    for (int q = 0; q < TA; ++q) {
#pragma unroll
        for (int t = 0; t < TB; ++t) S.u.Gp[warp][a0 + q][b0 + t] = acc[q][t];
        if (tb == 0) S.u.Gp[warp][a0 + q][F] = rh[q];
    }
    __syncthreads();
    float* dst = G_aug + (int64_t)w * F * (F + 1);
    const float reg = row_reg(n, p);
    for (int e = tid; e < F * (F + 1); e += kCtaThreads) {
        const int a = e / (F + 1), b = e % (F + 1);
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < kCtaWarps; ++q) v += S.u.Gp[q][a][b];
        if (a == b) v = (a < f) ? v + reg : 1.f;
        dst[e] = v;
    }
}

// ---------------------------------------------------------------------------
// Batched solve of augmented systems [G | b] (F x (F+1) each, padded rows are
// identity). Warp per system; rows[w] gives the output row, or w itself when
// rows is null.
template <int F>
__global__ void __launch_bounds__(256) k_solve_rows(const float* __restrict__ G_aug, const int32_t* __restrict__ rows,
                                                    int n_list, Params p, float* __restrict__ X_out,
                                                    int32_t* __restrict__ flags_out, Counters* cnt) {
    __shared__ float tile[8][F][F + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * 8 + warp;
    if (w >= n_list) return;
    const float* src = G_aug + (int64_t)w * F * (F + 1);
    for (int e = lane; e < F * (F + 1); e += 32) tile[warp][e / (F + 1)][e % (F + 1)] = src[e];
    __syncwarp();
    float v[F];
#pragma unroll
    for (int j = 0; j < F; ++j) v[j] = (lane < F) ? tile[warp][lane][j] : 0.f;
    const float rhs = (lane < F) ? tile[warp][lane][F] : 0.f;
    float x;
    int flags;
    float ratio;
    warp_solve<F>(v, rhs, p.f, p.gram_mode == GRAM_ASYM, p.ratio_max, x, flags, ratio);
    const int64_t i = rows ? (int64_t)rows[w] : (int64_t)w;
    if (lane < p.f) X_out[i * p.f + lane] = x;
    if (lane == 0) {
        if (flags_out) flags_out[i] = flags;
        record_flags(cnt, flags, ratio);
    }
}

// Pack f x f systems (plus rhs) from user buffers into the padded augmented layout.
template <int F>
__global__ void k_pack_aug(const float* __restrict__ G, const float* __restrict__ b, int64_t n_rows, int f,
                           float* __restrict__ G_aug) {
    const int64_t total = n_rows * F * (F + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = e / (F * (F + 1));
        const int r = (int)((e / (F + 1)) % F), c = (int)(e % (F + 1));
        float v;
        if (r >= f) v = (c == r) ? 1.f : 0.f;
        else if (c == F) v = b[w * f + r];
        else if (c >= f) v = 0.f;
        else v = G[(w * f + r) * f + c];
        G_aug[e] = v;
    }
}

// Unpack the augmented layout of listed rows into user buffers (f x f and f).
template <int F>
__global__ void k_unpack_aug(const float* __restrict__ G_aug, const int32_t* __restrict__ rows, int n_list, int f,
                             float* __restrict__ G, float* __restrict__ b) {
    const int64_t total = (int64_t)n_list * f * (f + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = e / (f * (f + 1));
        const int r = (int)((e / (f + 1)) % f), c = (int)(e % (f + 1));
        const int64_t i = rows[w];
        const float v = G_aug[(w * F + r) * (F + 1) + (c == f ? F : c)];
        if (c == f) b[i * f + r] = v;
        else G[(i * f + r) * f + c] = v;
    }
}

// ---------------------------------------------------------------------------
// Structure check of one side: indptr monotone from 0 to nnz, indices in
// range and strictly increasing inside each row, values finite.
// err bits: 1 = indptr, 2 = index range/order, 4 = non-finite value.
__global__ void k_validate(const int64_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                           const float* __restrict__ values, int64_t n_rows, int64_t n_cols, int64_t nnz,
                           unsigned* err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rows; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = indptr[i], b = indptr[i + 1];
        if (a < 0 || b < a || b > nnz || (i == 0 && a != 0) || (i == n_rows - 1 && b != nnz)) {
            atomicOr(err, 1u);
            continue;
        }
        int32_t prev = -1;
        for (int64_t e = a; e < b; ++e) {
            const int32_t j = indices[e];
            if (j <= prev || j >= n_cols) {
                atomicOr(err, 2u);
                break;
            }
            prev = j;
            const float v = values[e];
            if (!(fabsf(v) <= 3.402823466e38f)) atomicOr(err, 4u);
        }
    }
}

// ---------------------------------------------------------------------------
// Sum of squared errors over entries, FP32 dot products, FP64 sums in a
// fixed order: grid-stride partial per thread, block tree, then k_sum_partials.
constexpr int kEvalBlocks = 608;
constexpr int kEvalThreads = 256;

__global__ void __launch_bounds__(kEvalThreads) k_sse(int64_t n, const int32_t* __restrict__ iu,
                                                      const int32_t* __restrict__ im, const float* __restrict__ r,
                                                      const float* __restrict__ U, const float* __restrict__ M, int f,
                                                      double* __restrict__ partials) {
    __shared__ double red[kEvalThreads];
    double acc = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)kEvalThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kEvalThreads) {
        const float* u = U + (int64_t)iu[e] * f;
        const float* m = M + (int64_t)im[e] * f;
        float d = 0.f;
        for (int a = 0; a < f; ++a) d = fmaf(u[a], m[a], d);
        const double res = (double)r[e] - (double)d;
        acc += res * res;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kEvalThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double* __restrict__ partials, int n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < n; ++q) s += partials[q];
        *out = s;
    }
}

__global__ void k_zero_rows(const int32_t* __restrict__ rows, int n_list, int f, float* __restrict__ X_out) {
    const int64_t total = (int64_t)n_list * f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        X_out[(int64_t)rows[e / f] * f + e % f] = 0.f;
}

}  // namespace als
