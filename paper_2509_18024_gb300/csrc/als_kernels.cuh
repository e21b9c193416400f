// Kernels of one Core-ALS half-sweep on CUDA cores (FP32), n_f <= 32.
//
// Rows are bucketed by length by the host planner:
//   * k_warp_rows  : n_i <= 32. One warp per row does CES (Algorithm 1) and
//                    the Gram assembly of Eq. (core_ui) in registers and a
//                    warp-private shared-memory tile.
//   * k_cta_rows   : 32 < n_i <= 1024 (three capacity buckets). One CTA per
//                    row stages the slice in shared memory once, selects by
//                    an exact radix select and assembles the masked Gram.
//   * k_split_*    : n_i > 1024. The row is cut into 512-element chunks, one
//                    CTA each; the radix passes meet in per-row global
//                    histograms and the chunk Grams are summed in chunk order.
//   The augmented systems [G | b] of all rows are solved by one batched
//   k_solve_rows launch (warp per system).
#pragma once

#include "als_device.cuh"

namespace als {

constexpr int kWarpRowMax = 32;

// ---------------------------------------------------------------------------
// Warp per row (n_i <= 32): gather, CES and the masked Gram of the row; the
// augmented system [G | b] (regulariser added, padding rows identity) is
// solved by the same warp into X_out (flags, counters and FP64 redo list as
// k_solve_rows), or, with X_out null, goes to G_aug[w]. masks_only: stop
// after the masks.
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
__global__ void __launch_bounds__(256, 3) k_warp_rows(Side side, Params p, const int32_t* __restrict__ rows,
                                                   int n_list, bool masks_only, uint32_t* __restrict__ masks_out,
                                                   float* __restrict__ G_aug, float* __restrict__ X_out,
                                                   int32_t* __restrict__ flags_out, Counters* cnt, Fallback fb) {
    __shared__ WarpRowTile<F> tiles[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * 8 + warp;
    if (w >= n_list) return;
    WarpRowTile<F>& T = tiles[warp];
    const int f = p.f;
    const int64_t i = rows[w];
    const int64_t lo = side.indptr[i];
    const int n = min((int)(side.indptr[i + 1] - lo), kWarpRowMax);  // the plan's bound

    if (lane < n) {
        T.idx[lane] = factor_row(side.indices[lo + lane], side.n_cols);
        T.r[lane] = side.values[lo + lane];
    }
    __syncwarp();
    for (int e = lane; e < n * F; e += 32) {
        const int k = e / F, a = e % F;
        T.u.x[k][a] = (a < f) ? __ldg(side.Y + (int64_t)T.idx[k] * f + a) : 0.f;
    }
    __syncwarp();

    if (p.gP != nullptr) {
        // Fast variant: the factor-wide keep rule, positions = rows of Y.
        const int32_t j = lane < n ? T.idx[lane] : 0;
        for (int a = 0; a < F; ++a) {
            const bool kp = a < f && lane < n && keep_rule(mag_key(T.u.x[lane][a]), p.gP[a], p.gMk[a], j, p.gcut[a]);
            const unsigned m = __ballot_sync(kFull, kp);
            if (lane == 0) T.sel[a] = m;
        }
    } else {
        const int s = (int)row_budget(n, p);
        for (int a = 0; a < F; ++a) {
            unsigned m = 0u;
            if (a < f) {
                uint32_t key = (lane < n) ? mag_key(T.u.x[lane][a]) : 0u;
                m = warp_ces_column(key, n, s);
            }
            if (lane == 0) T.sel[a] = m;
        }
    }
    __syncwarp();
    if (masks_out != nullptr && lane < n) {
        uint32_t word = 0u;
        for (int a = 0; a < f; ++a) word |= ((T.sel[a] >> lane) & 1u) << a;
        masks_out[lo + lane] = word;
    }
    if (masks_only) return;

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
    if (X_out == nullptr) {
        float* dst = G_aug + (int64_t)w * F * (F + 1);
        for (int e = lane; e < F * (F + 1); e += 32) dst[e] = T.u.G[e / (F + 1)][e % (F + 1)];
        return;
    }
    // The system never leaves the SM: the warp solves it here, exactly as
    // k_solve_rows does from the stored copy.
    float v[F];
#pragma unroll
    for (int j = 0; j < F; ++j) v[j] = (lane < F) ? T.u.G[lane][j] : 0.f;
    const float rhs = (lane < F) ? T.u.G[lane][F] : 0.f;
    float x;
    int flags;
    float ratio;
    warp_solve<F>(v, rhs, p.f, p.gram_mode == GRAM_ASYM, p.ratio_max, x, flags, ratio);
    if (lane < p.f) X_out[i * p.f + lane] = x;
    if (lane == 0) {
        if (flags_out) flags_out[i] = flags;
        record_flags(cnt, flags, ratio);
        fallback_push(fb, flags, i);
    }
}

}  // namespace als

#include "als_rows.cuh"

namespace als {

// ---------------------------------------------------------------------------
// Batched solve of augmented systems [G | b] (F x (F+1) each, padded rows are
// identity). Warp per system; rows[w] gives the output row, or w itself when
// rows is null.
template <int F>
__global__ void __launch_bounds__(256, 4) k_solve_rows(const float* __restrict__ G_aug, const int32_t* __restrict__ rows,
                                                    int n_list, Params p, float* __restrict__ X_out,
                                                    int32_t* __restrict__ flags_out, Counters* cnt, Fallback fb) {
    __shared__ __align__(16) float tile[8][F][F + 1];
    __shared__ __align__(8) uint64_t bar[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * 8 + warp;
    if (w >= n_list) return;
    const float* src = G_aug + (int64_t)w * F * (F + 1);
    float* t = &tile[warp][0][0];  // the tile is contiguous with the same layout
    if (!stage_warp(t, src, F * (F + 1), &bar[warp], p.err)) {
        for (int e = lane; e < F * (F + 1); e += 32) t[e] = 0.f;  // a copy that never completed
        __syncwarp();
    }
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
        fallback_push(fb, flags, i);
    }
}

// CTA-wide elimination on an augmented system A = [G | b] (F x (F+1), type T,
// shared memory), rows >= f padding: right-looking with partial pivoting
// (`pivot`) or diagonal pivots, then column-oriented back substitution into
// xs. All threads of the CTA call it. Returns flags; ratio = max/min pivot
// over the first f pivots.
template <typename T, int F>
__device__ __forceinline__ int cta_lu_solve(T (*A)[F + 1], T* xs, int* s_piv, int f, bool pivot, float ratio_max,
                                            float& ratio_out) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nt = blockDim.x;
    T pmax = 0, pmin = (T)INFINITY;
    bool singular = false;
    for (int k = 0; k < F; ++k) {
        if (warp == 0) {
            int bi = k;
            if (pivot) {
                T best = -1;
                bi = F;
                for (int i = k + lane; i < F; i += 32) {
                    const T v = A[i][k] < 0 ? -A[i][k] : A[i][k];
                    if (v > best) {
                        best = v;
                        bi = i;
                    }
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    const T ob = __shfl_xor_sync(kFull, best, o);
                    const int oi = __shfl_xor_sync(kFull, bi, o);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                }
            }
            if (lane == 0) *s_piv = bi;
        }
        __syncthreads();
        const int pr = *s_piv;
        if (pr != k)
            for (int j = k + tid; j <= F; j += nt) {
                const T t = A[k][j];
                A[k][j] = A[pr][j];
                A[pr][j] = t;
            }
        __syncthreads();
        const T pv = A[k][k];
        const T apv = pivot ? (pv < 0 ? -pv : pv) : pv;
        if (k < f) {
            if (!(apv > 0)) singular = true;
            pmax = apv > pmax ? apv : pmax;
            pmin = apv < pmin ? apv : pmin;
        }
        if (pv != (T)0) {
            for (int i = k + 1 + tid; i < F; i += nt) A[i][k] /= pv;
            __syncthreads();
            const int cols = F - k;  // columns k+1 .. F (rhs included)
            const int total = (F - 1 - k) * cols;
            for (int e = tid; e < total; e += nt) {
                const int i = k + 1 + e / cols, j = k + 1 + e % cols;
                A[i][j] -= A[i][k] * A[k][j];
            }
        }
        __syncthreads();
    }
    for (int k = F - 1; k >= 0; --k) {
        if (tid == 0) xs[k] = A[k][F] / A[k][k];
        __syncthreads();
        const T xk = xs[k];
        for (int i = tid; i < k; i += nt) A[i][F] -= A[i][k] * xk;
        __syncthreads();
    }
    int flags = 0;
    ratio_out = (f > 0) ? (float)(pmax / pmin) : 1.f;
    if (singular) {
        flags = FLAG_SINGULAR | FLAG_RATIO;
        ratio_out = __int_as_float(0x7f800000);
    } else if (!(ratio_out <= ratio_max)) {
        flags = FLAG_RATIO;
    }
    return flags;
}

// Correction solve of a refinement step at F = 64, 128: forward and back
// substitution with the factors a previous solve stored (row i of the block:
// multipliers before its own pivot step, U from it on; the new rhs in column
// F, physical row order; perm_buf: the physical row of each step). One warp
// per system: the block (pitch F + 1) comes into shared memory with one bulk
// copy, lane holds logical rows lane + 32 s; the forward pass takes the
// steps in order and the back pass in reverse. A bulk copy whose bounded wait ran out
// leaves a zero correction (and bit 0 of the error word).
template <int F>
__global__ void __launch_bounds__(32) k_solve_replay(const float* __restrict__ G_aug,
                                                     const int32_t* __restrict__ rows, int n_list, Params p,
                                                     float* __restrict__ X_out,
                                                     const int32_t* __restrict__ perm_buf) {
    constexpr int S = F / 32;
    extern __shared__ __align__(16) float smem_f[];  // F x (F + 1)
    __shared__ __align__(8) uint64_t bar;
    __shared__ float dinv[F];
    const int lane = threadIdx.x;
    const int w = blockIdx.x;
    if (w >= n_list) return;
    const bool staged = stage_warp(smem_f, G_aug + (int64_t)w * F * (F + 1), F * (F + 1), &bar, p.err);
    int pr[S];
    float y[S];
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
        pr[s2] = min(max(perm_buf[(int64_t)w * F + lane + 32 * s2], 0), F - 1);
        y[s2] = smem_f[pr[s2] * (F + 1) + F];
        const float ukk = smem_f[pr[s2] * (F + 1) + lane + 32 * s2];
        dinv[lane + 32 * s2] = ukk != 0.f ? 1.0f / ukk : 0.f;
    }
    __syncwarp();
    // Forward: y_i -= l_ik y_k for logical i > k (unit lower factor).
#pragma unroll 4
    for (int k = 0; k < F; ++k) {
        const float yk = __shfl_sync(kFull, y[k / 32], k % 32);
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2)
            if (lane + 32 * s2 > k) y[s2] = fmaf(-smem_f[pr[s2] * (F + 1) + k], yk, y[s2]);
    }
    const int64_t i = rows ? (int64_t)rows[w] : (int64_t)w;
    float* xo = X_out + i * p.f;
#pragma unroll 4
    for (int k = F - 1; k >= 0; --k) {
        const float yk = __shfl_sync(kFull, y[k / 32], k % 32);
        const float xk = yk * dinv[k];
        if (lane == k % 32 && k < p.f) xo[k] = staged ? xk : 0.f;
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2)
            if (lane + 32 * s2 < k) y[s2] = fmaf(-smem_f[pr[s2] * (F + 1) + k], xk, y[s2]);
    }
}

// Register-resident LU for widths above 32: one thread per matrix row, the row
// (F + 1 values with the rhs) in registers. Columns are eliminated in blocks
// of 8 steps; between blocks every row shifts its registers left by 8, so
// that the pivot column of step s of a block is always register s (all
// register indices are compile-time). Step k: every live row offers |a_ik|
// (warp max + lowest row), the pivot is the largest over the CTA (lowest row
// on ties; row k itself for the symmetric modes), its row is published as
// float4s into U[k] (shared memory, U in step order), and every live row
// subtracts l_ik U[k] with l_ik = a_ik / u_kk, keeping l_ik in the dead
// register. At n_f = 128 a step updates only the block's own 8 columns and
// the trailing columns take the block's 8 updates together afterwards
// (reg_lu_block); the results are the same bit for bit, and the deferred
// form needs 168 registers, so three CTAs share an SM. One warp
// back-substitutes from U. Rows never move (partial pivoting through the
// step order). The system comes into shared memory with one bulk copy.
// store != 0: each row's block of L / U entries goes back to G_aug (L before
// the row's own pivot step, U from it on) and the physical row of each step
// to perm_buf, the form k_solve_replay reads.
template <int F>
struct RegSolve {
    static constexpr int NT = F;      // threads per system
    static constexpr int NW = F / 32;
    static constexpr int R = F + 1;   // registers per row (with the rhs)
    static constexpr int P = F + 4;   // U row pitch (floats)
    static constexpr int NCH = (R + 3) / 4;
    static constexpr size_t SMEM = (size_t)F * P * sizeof(float);
};

// One block of 8 elimination steps of k_solve_reg (block t: columns 8t ..
// 8t + 7 in registers 0..7), then the left shift by 8. NCHB bounds the float4
// chunks that can still hold live columns in this block (compile-time, so
// that later blocks skip the dead tail without runtime tests).
// The steps update only the block's own 8 columns; the trailing columns
// (and the rhs) take the block's 8 updates afterwards in one pass with no
// barrier between them. Each pivot row publishes its trailing part as it
// stands, and a triangular solve with a thread per trailing column (the
// earlier steps' multiples of the published rows taken off in step order)
// turns those into the U rows, so every product and its place in each sum
// are those of eliminating one step at a time.
template <int F, int NCHB>
__device__ __forceinline__ void reg_lu_block(float (&r)[F + 1], const int t, bool& live, const bool pivot,
                                             float (*U)[F + 4], uint32_t (*s_key)[F / 32], int (*s_idx)[F / 32],
                                             float* s_pv, float* s_dinv, int* s_ord, const int store, float* src) {
    constexpr int NW = F / 32, R = F + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rem = R - 8 * t;  // registers still holding columns 8t .. F
    int own = -1;  // the step of this block at which this row is the pivot
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int k = 8 * t + s;
        uint32_t key;
        if (pivot) key = live ? __float_as_uint(fabsf(r[s])) + 1u : 0u;
        else key = tid == k ? 1u : 0u;
        const uint32_t m = __reduce_max_sync(kFull, key);
        const unsigned bal = __ballot_sync(kFull, key == m && m != 0u);
        if (lane == 0) {
            s_key[k & 1][warp] = m;
            s_idx[k & 1][warp] = bal ? warp * 32 + __ffs(bal) - 1 : F;
        }
        __syncthreads();
        uint32_t bm = 0u;
        int pidx = F;
#pragma unroll
        for (int v = 0; v < NW; ++v) {
            const uint32_t kv = s_key[k & 1][v];
            const int iv = s_idx[k & 1][v];
            if (kv > bm || (kv == bm && iv < pidx)) {
                bm = kv;
                pidx = iv;
            }
        }
        if (tid == pidx) {
            float* urow = &U[k][8 * t];
#pragma unroll
            for (int c = 0; c < NCHB; ++c) {
                if (4 * c < rem) {
                    if (4 * c + 3 < R) {
                        *reinterpret_cast<float4*>(urow + 4 * c) = make_float4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (4 * c + e < R) urow[4 * c + e] = r[4 * c + e];
                    }
                }
            }
            const float pv = r[s];
            s_pv[k] = pv;
            s_dinv[k] = pv != 0.f ? 1.0f / pv : 0.f;
            s_ord[k] = tid;
            live = false;
            own = s;
        }
        __syncthreads();
        const float di = s_dinv[k];
        if (live && di != 0.f) {
            const float l = r[s] * di;
            r[s] = l;
            const float* urow = &U[k][8 * t];
#pragma unroll
            for (int j = s + 1; j < 8; ++j) r[j] = fmaf(-l, urow[j], r[j]);
        }
    }
    // U rows of the block's steps, trailing columns (rhs included): thread
    // tid takes column 8t + 8 + tid. The published rows read here were all
    // written before the last step's barrier; the block's own columns, which
    // the last step's updates read, are not touched.
    if (8 + tid < rem) {
        const int col = 8 * t + 8 + tid;
        float u[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) u[s] = U[8 * t + s][col];
#pragma unroll
        for (int s = 0; s < 7; ++s) {
            if (s_dinv[8 * t + s] != 0.f) {
#pragma unroll
                for (int s2 = s + 1; s2 < 8; ++s2) u[s2] = fmaf(-U[8 * t + s2][8 * t + s], u[s], u[s2]);
            }
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) U[8 * t + s][col] = u[s];
    }
    __syncthreads();
    if (live) {
        // The block's 8 updates of the trailing columns: chunk by chunk, each
        // element taking the steps in order.
        float l[8];
        bool use[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            use[s] = s_dinv[8 * t + s] != 0.f;
            l[s] = r[s];
        }
#pragma unroll
        for (int c = 2; c < NCHB; ++c) {
            if (4 * c < rem) {
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    if (!use[s]) continue;
                    const float* urow = &U[8 * t + s][8 * t];
                    float u4[4];
                    if (4 * c + 3 < R) {
                        const float4 v = *reinterpret_cast<const float4*>(urow + 4 * c);
                        u4[0] = v.x;
                        u4[1] = v.y;
                        u4[2] = v.z;
                        u4[3] = v.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) u4[e] = (4 * c + e < R) ? urow[4 * c + e] : 0.f;
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = 4 * c + e;
                        if (j < R) r[j] = fmaf(-l[s], u4[e], r[j]);
                    }
                }
            }
        }
    } else if (store && own >= 0) {
        // This block's pivot rows take their finished U entries back, so that
        // the later blocks store them.
        const float* urow = &U[8 * t + own][8 * t];
#pragma unroll
        for (int c = 2; c < NCHB; ++c)
            if (4 * c < rem)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * c + e < R) r[4 * c + e] = urow[4 * c + e];
    }
    if (store) {
        float* dst = src + (int64_t)tid * (F + 1) + 8 * t;
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[e] = r[e];
    }
#pragma unroll
    for (int j = 0; j + 8 < R; ++j) r[j] = r[j + 8];
}

// n_f = 64 form of reg_lu_block: every step updates the whole remaining
// row at once (the deferred trailing update does not pay at this width).
template <int F, int NCHB>
__device__ __forceinline__ void reg_lu_steps(float (&r)[F + 1], const int t, bool& live, const bool pivot,
                                             float (*U)[F + 4], uint32_t (*s_key)[F / 32], int (*s_idx)[F / 32],
                                             float* s_pv, float* s_dinv, int* s_ord, const int store, float* src) {
    constexpr int NW = F / 32, R = F + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rem = R - 8 * t;  // registers still holding columns 8t .. F
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int k = 8 * t + s;
        uint32_t key;
        if (pivot) key = live ? __float_as_uint(fabsf(r[s])) + 1u : 0u;
        else key = tid == k ? 1u : 0u;
        const uint32_t m = __reduce_max_sync(kFull, key);
        const unsigned bal = __ballot_sync(kFull, key == m && m != 0u);
        if (lane == 0) {
            s_key[k & 1][warp] = m;
            s_idx[k & 1][warp] = bal ? warp * 32 + __ffs(bal) - 1 : F;
        }
        __syncthreads();
        uint32_t bm = 0u;
        int pidx = F;
#pragma unroll
        for (int v = 0; v < NW; ++v) {
            const uint32_t kv = s_key[k & 1][v];
            const int iv = s_idx[k & 1][v];
            if (kv > bm || (kv == bm && iv < pidx)) {
                bm = kv;
                pidx = iv;
            }
        }
        if (tid == pidx) {
            float* urow = &U[k][8 * t];
#pragma unroll
            for (int c = 0; c < NCHB; ++c) {
                if (4 * c < rem) {
                    if (4 * c + 3 < R) {
                        *reinterpret_cast<float4*>(urow + 4 * c) = make_float4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (4 * c + e < R) urow[4 * c + e] = r[4 * c + e];
                    }
                }
            }
            const float pv = r[s];
            s_pv[k] = pv;
            s_dinv[k] = pv != 0.f ? 1.0f / pv : 0.f;
            s_ord[k] = tid;
            live = false;
        }
        __syncthreads();
        const float di = s_dinv[k];
        if (live && di != 0.f) {
            const float l = r[s] * di;
            r[s] = l;
            const float* urow = &U[k][8 * t];
#pragma unroll
            for (int c = (s + 1) / 4; c < NCHB; ++c) {
                if (4 * c < rem) {
                    float u4[4];
                    if (4 * c + 3 < R) {
                        const float4 v = *reinterpret_cast<const float4*>(urow + 4 * c);
                        u4[0] = v.x;
                        u4[1] = v.y;
                        u4[2] = v.z;
                        u4[3] = v.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) u4[e] = (4 * c + e < R) ? urow[4 * c + e] : 0.f;
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = 4 * c + e;
                        if (j > s && j < R) r[j] = fmaf(-l, u4[e], r[j]);
                    }
                }
            }
        }
    }
    if (store) {
        float* dst = src + (int64_t)tid * (F + 1) + 8 * t;
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[e] = r[e];
    }
#pragma unroll
    for (int j = 0; j + 8 < R; ++j) r[j] = r[j + 8];
}

template <int F>
__global__ void __launch_bounds__(RegSolve<F>::NT, F == 64 ? 8 : 3) k_solve_reg(
    float* __restrict__ G_aug, const int32_t* __restrict__ rows, int n_list, Params p, float* __restrict__ X_out,
    int32_t* __restrict__ flags_out, Counters* cnt, Fallback fb, int32_t* __restrict__ perm_buf, int store) {
    using C = RegSolve<F>;
    constexpr int NW = C::NW, R = C::R, P = C::P;
    extern __shared__ __align__(16) float smem_f[];
    float (*U)[P] = reinterpret_cast<float (*)[P]>(smem_f);
    __shared__ uint32_t s_key[2][NW];
    __shared__ int s_idx[2][NW];
    __shared__ float s_dinv[F];
    __shared__ float s_pv[F];
    __shared__ int s_ord[F];
    __shared__ __align__(8) uint64_t bar_ld;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w = blockIdx.x;
    if (w >= n_list) return;
    float* src = G_aug + (int64_t)w * F * (F + 1);
    // Stage the system (row-major, pitch F + 1) in the U area with one bulk
    // copy, then each thread takes its row.
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_ld)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t ld_phase = 0u;
    const bool staged = stage_block(smem_f, src, F * (F + 1), &bar_ld, ld_phase, p.err);
    float r[R];
#pragma unroll
    for (int j = 0; j < R; ++j) r[j] = smem_f[tid * (F + 1) + j];
    __syncthreads();
    const bool pivot = p.gram_mode == GRAM_ASYM;
    bool live = true;
    // n_f = 128: four quarters of the elimination, each with the chunk bound
    // of its first block (the live width shrinks by 8 columns per block). At
    // n_f = 64 one bound for all blocks keeps the kernel within its registers.
    constexpr int QB = F / 32;  // blocks per quarter
    if constexpr (F < 128) {
        for (int t = 0; t < F / 8; ++t)
            reg_lu_steps<F, (R + 3) / 4>(r, t, live, pivot, U, s_key, s_idx, s_pv, s_dinv, s_ord, store, src);
    } else {
    for (int t = 0; t < QB; ++t)
        reg_lu_block<F, (R + 3) / 4>(r, t, live, pivot, U, s_key, s_idx, s_pv, s_dinv, s_ord, store, src);
    for (int t = QB; t < 2 * QB; ++t)
        reg_lu_block<F, (R - 8 * QB + 3) / 4>(r, t, live, pivot, U, s_key, s_idx, s_pv, s_dinv, s_ord, store, src);
    for (int t = 2 * QB; t < 3 * QB; ++t)
        reg_lu_block<F, (R - 16 * QB + 3) / 4>(r, t, live, pivot, U, s_key, s_idx, s_pv, s_dinv, s_ord, store, src);
    for (int t = 3 * QB; t < 4 * QB; ++t)
        reg_lu_block<F, (R - 24 * QB + 3) / 4>(r, t, live, pivot, U, s_key, s_idx, s_pv, s_dinv, s_ord, store, src);
    }
    __syncthreads();
    bool singular = false;
    float pmax = 0.f, pmin = __int_as_float(0x7f800000);
    if (tid == 0)
        for (int k = 0; k < p.f; ++k) {
            const float apv = pivot ? fabsf(s_pv[k]) : s_pv[k];
            if (!(apv > 0.f)) singular = true;
            pmax = fmaxf(pmax, apv);
            pmin = fminf(pmin, apv);
        }
    // Back substitution by warp 0 on U (rows in step order): lane holds
    // steps lane + 32 s2.
    if (warp == 0) {
        constexpr int S = F / 32;
        float y[S];
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) y[s2] = U[lane + 32 * s2][F];
        const int64_t i = rows ? (int64_t)rows[w] : (int64_t)w;
        float* xo = X_out + i * p.f;
        const bool sing = __shfl_sync(kFull, (int)singular, 0) != 0 || !staged;
#pragma unroll
        for (int k = F - 1; k >= 0; --k) {
            const float yk = __shfl_sync(kFull, y[k / 32], k % 32);
            const float xk = yk * s_dinv[k];
            if (lane == k % 32 && k < p.f) xo[k] = sing ? 0.f : xk;
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2)
                if (lane + 32 * s2 < k) y[s2] = fmaf(-U[lane + 32 * s2][k], xk, y[s2]);
        }
    }
    if (store)
        for (int k = tid; k < F; k += F) perm_buf[(int64_t)w * F + k] = s_ord[k];
    if (tid == 0) {
        int flags = 0;
        float ratio = (p.f > 0) ? pmax / pmin : 1.f;
        if (singular) {
            flags = FLAG_SINGULAR | FLAG_RATIO;
            ratio = __int_as_float(0x7f800000);
        } else if (!(ratio <= p.ratio_max)) {
            flags = FLAG_RATIO;
        }
        const int64_t i = rows ? (int64_t)rows[w] : (int64_t)w;
        if (flags_out) flags_out[i] = flags;
        record_flags(cnt, flags, ratio);
        fallback_push(fb, flags, i);
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
// Entry-parallel: an entry whose index does not exceed its predecessor's must
// start a row, which a binary search of indptr decides (bounded by log2 of
// the row count even when indptr itself is malformed).
__global__ void k_validate(const int64_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                           const float* __restrict__ values, int64_t n_rows, int64_t n_cols, int64_t nnz,
                           unsigned* err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned bad = 0u;
    for (int64_t i = t0; i < n_rows; i += stride) {
        const int64_t a = indptr[i], b = indptr[i + 1];
        if (a < 0 || b < a || b > nnz || (i == 0 && a != 0) || (i == n_rows - 1 && b != nnz)) bad |= 1u;
    }
    for (int64_t e = t0; e < nnz; e += stride) {
        const int32_t j = indices[e];
        if (j < 0 || j >= n_cols) bad |= 2u;
        if (!(fabsf(values[e]) <= 3.402823466e38f)) bad |= 4u;
        if (e > 0 && j <= indices[e - 1]) {
            int64_t lo = 0, hi = n_rows;  // first i with indptr[i] >= e
            for (int it = 0; it < 64 && lo < hi; ++it) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (indptr[mid] < e) lo = mid + 1;
                else hi = mid;
            }
            if (indptr[lo] != e) bad |= 2u;
        }
    }
    if (bad) atomicOr(err, bad);
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
    // 16-byte loads when rows are whole float4s (the sum order is a = 0..f-1 either way).
    const bool vec = (f % 4) == 0 && ((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(M)) & 15u) == 0;
    for (int64_t e = blockIdx.x * (int64_t)kEvalThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kEvalThreads) {
        const float* u = U + (int64_t)iu[e] * f;
        const float* m = M + (int64_t)im[e] * f;
        float d = 0.f;
        if (vec) {
            for (int a = 0; a < f; a += 4) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(u + a));
                const float4 y = __ldg(reinterpret_cast<const float4*>(m + a));
                d = fmaf(x.x, y.x, d);
                d = fmaf(x.y, y.y, d);
                d = fmaf(x.z, y.z, d);
                d = fmaf(x.w, y.w, d);
            }
        } else {
            for (int a = 0; a < f; ++a) d = fmaf(u[a], m[a], d);
        }
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

// One warp: lane l sums partials l, l + 32, ... in order, then a fixed
// butterfly adds the lanes (the same order every run).
__global__ void k_sum_partials(const double* __restrict__ partials, int n, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    double s = 0.0;
    for (int q = lane; q < n; q += 32) s += partials[q];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) *out = s;
}

__global__ void k_zero_rows(const int32_t* __restrict__ rows, int n_list, int f, float* __restrict__ X_out) {
    const int64_t total = (int64_t)n_list * f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        X_out[(int64_t)rows[e / f] * f + e % f] = 0.f;
}

}  // namespace als
