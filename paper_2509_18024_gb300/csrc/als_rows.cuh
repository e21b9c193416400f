// CTA-resident rows (32 < n_i <= 1024) and split rows (n_i > 1024) of one
// Core-ALS half-sweep: CES (Algorithm 1) by exact radix select, then the
// masked Gram of Eq. (core_ui) in FP32 on CUDA cores.
#pragma once

#include "als_device.cuh"

namespace als {

constexpr int kCtaThreads = 256;
constexpr int kCtaWarps = kCtaThreads / 32;
constexpr int kSplitChunk = 512;  // elements per chunk of a split row
constexpr int kSplitMin = 1024;   // rows longer than this are split

// ---------------------------------------------------------------------------
// Masked Gram of a staged tile, warps split the positions, lanes tile [G|b]:
// G[a][b] += w_ka x_ka w'_kb x_kb, rhs[a] += w_ka x_ka r_k.
template <int F>
struct GramAcc {
    static constexpr int TA = F / 8, TB = F / 4;
    float acc[TA][TB];
    float rh[TA];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < TA; ++q) {
            rh[q] = 0.f;
#pragma unroll
            for (int t = 0; t < TB; ++t) acc[q][t] = 0.f;
        }
    }
    // x: [*][F] row-major tile, mask: keep bits per position, r: ratings.
    __device__ __forceinline__ void add_tile(const float (*x)[F], const uint32_t* mask, const float* r, int k_begin,
                                             int k_end, int k_step, bool sym) {
        const int lane = threadIdx.x & 31;
        const int a0 = (lane >> 2) * TA, b0 = (lane & 3) * TB;
        for (int k = k_begin; k < k_end; k += k_step) {
            const uint32_t m = mask[k];
            float xa[TA], xb[TB];
#pragma unroll
            for (int q = 0; q < TA; ++q) xa[q] = ((m >> (a0 + q)) & 1u) ? x[k][a0 + q] : 0.f;
#pragma unroll
            for (int t = 0; t < TB; ++t) xb[t] = (!sym || ((m >> (b0 + t)) & 1u)) ? x[k][b0 + t] : 0.f;
            const float rk = r[k];
#pragma unroll
            for (int q = 0; q < TA; ++q) {
                rh[q] = fmaf(xa[q], rk, rh[q]);
#pragma unroll
                for (int t = 0; t < TB; ++t) acc[q][t] = fmaf(xa[q], xb[t], acc[q][t]);
            }
        }
    }
    __device__ __forceinline__ void store(float (*Gp)[F + 1]) const {
        const int lane = threadIdx.x & 31;
        const int a0 = (lane >> 2) * TA, b0 = (lane & 3) * TB;
#pragma unroll
        for (int q = 0; q < TA; ++q) {
#pragma unroll
            for (int t = 0; t < TB; ++t) Gp[a0 + q][b0 + t] = acc[q][t];
            if ((lane & 3) == 0) Gp[a0 + q][F] = rh[q];
        }
    }
};

// Stage positions [0, cn) of the slice starting at absolute entry e0.
template <int F>
__device__ __forceinline__ void stage_tile(float (*x)[F], float* r, int32_t* idx, const Side& side, int f,
                                           int64_t e0, int cn) {
    for (int k = threadIdx.x; k < cn; k += kCtaThreads) {
        idx[k] = side.indices[e0 + k];
        r[k] = side.values[e0 + k];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cn * F; e += kCtaThreads) {
        const int k = e / F, a = e % F;
        x[k][a] = (a < f) ? __ldg(side.Y + (int64_t)idx[k] * f + a) : 0.f;
    }
    __syncthreads();
}

// Selection state of one column before any pass: keep nothing (padding,
// s = 0), everything (s >= n), or open.
__device__ __forceinline__ void init_column(int a, int f, long long s, long long n, uint32_t& P, uint32_t& Mk,
                                            int& need, int& cut, int& done) {
    need = (int)s;
    cut = 0x7fffffff;
    P = 0u;
    Mk = 0u;
    done = 0;
    if (a >= f || s == 0) {
        P = 0xffffffffu;
        Mk = 0xffffffffu;
        cut = 0;
        done = 1;
    } else if (s >= n) {
        done = 1;
    }
}

// ---------------------------------------------------------------------------
// CTA per row, slice resident in shared memory (n_i <= NS).
template <int F, int NS>
struct CtaSmem {
    float x[NS][F];
    float r[NS];
    int32_t idx[NS];
    uint32_t mask[NS];
    union {
        uint32_t hist[F][256];
        float Gp[kCtaWarps][F][F + 1];
    } u;
    uint32_t P[F];
    uint32_t Mk[F];
    int32_t need[F];
    int32_t cut[F];
    int32_t done[F];
    int32_t active;
};

// mode 0/1: write the augmented system of list entry w to G_aug[w]; mode 2:
// masks only.
template <int F, int NS>
__global__ void __launch_bounds__(kCtaThreads) k_cta_rows(Side side, Params p, const int32_t* __restrict__ rows,
                                                          int n_list, int mode, float* __restrict__ G_aug,
                                                          uint32_t* __restrict__ masks_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem<F, NS>& S = *reinterpret_cast<CtaSmem<F, NS>*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w = blockIdx.x;
    if (w >= n_list) return;
    const int f = p.f;
    const int64_t i = rows[w];
    const int64_t lo = side.indptr[i];
    const int n = (int)(side.indptr[i + 1] - lo);
    const long long s = row_budget(n, p);
    const int a_t = tid % F;  // thread t always handles column t mod F
    const int k0 = tid / F;
    constexpr int kstep = kCtaThreads / F;

    if (tid < F) {
        uint32_t P, Mk;
        int need, cut, done;
        init_column(tid, f, s, n, P, Mk, need, cut, done);
        S.P[tid] = P;
        S.Mk[tid] = Mk;
        S.need[tid] = need;
        S.cut[tid] = cut;
        S.done[tid] = done;
    }
    if (tid == 0) S.active = (f > 0 && s > 0 && s < n) ? 1 : 0;
    stage_tile<F>(S.x, S.r, S.idx, side, f, lo, n);

    for (int pass = 0; pass < 4; ++pass) {
        if (!S.active) break;
        const uint32_t hm = radix_before(pass);
        for (int e = tid; e < F * 256; e += kCtaThreads) (&S.u.hist[0][0])[e] = 0u;
        __syncthreads();
        if (!S.done[a_t]) {
            const uint32_t Pa = S.P[a_t];
            for (int k = k0; k < n; k += kstep) {
                const uint32_t key = mag_key(S.x[k][a_t]);
                if ((key & hm) == Pa) atomicAdd(&S.u.hist[a_t][radix_digit(key, pass)], 1u);
            }
        }
        __syncthreads();
        for (int a = warp; a < F; a += kCtaWarps) {
            if (S.done[a]) continue;
            const BinPick bp = warp_pick_bin(S.u.hist[a], (uint32_t)S.need[a]);
            if (lane == 0) {
                S.P[a] |= (uint32_t)bp.digit << radix_shift(pass);
                S.Mk[a] = radix_after(pass);
                S.need[a] = (int)bp.newneed;
                if (bp.inbin == bp.newneed) S.done[a] = 1;
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
    // Open columns: the full key P has more copies than places left; keep the
    // lowest positions.
    for (int a = warp; a < F; a += kCtaWarps) {
        if (S.done[a]) continue;
        const uint32_t T = S.P[a];
        const int nd = S.need[a];
        int seen = 0, cut = n;
        for (int kb = 0; kb < n; kb += 32) {
            const int k = kb + lane;
            const bool eq = k < n && mag_key(S.x[k][a]) == T;
            unsigned b = __ballot_sync(kFull, eq);
            const int c = __popc(b);
            if (seen + c >= nd) {
                int want = nd - seen;
                while (--want > 0) b &= b - 1u;
                cut = kb + __ffs(b);
                break;
            }
            seen += c;
        }
        if (lane == 0) S.cut[a] = cut;
    }
    __syncthreads();

    const uint32_t Pa = S.P[a_t], Ma = S.Mk[a_t];
    const int cuta = S.cut[a_t];
    const uint32_t fmask = (F == 32) ? kFull : ((1u << F) - 1u);
    for (int kk = 0; kk < n; kk += kstep) {
        const int k = kk + k0;
        const bool keep = k < n && keep_rule(mag_key(S.x[k][a_t]), Pa, Ma, k, cuta);
        const unsigned b = __ballot_sync(kFull, keep);
        if (a_t == 0 && k < n) S.mask[k] = (b >> (lane & ~(F - 1))) & fmask;
    }
    __syncthreads();
    if (masks_out != nullptr)
        for (int k = tid; k < n; k += kCtaThreads) masks_out[lo + k] = S.mask[k];
    if (mode == 2) return;
    GramAcc<F> g;
    g.zero();
    g.add_tile(S.x, S.mask, S.r, warp, n, kCtaWarps, p.gram_mode == GRAM_SYM);
    g.store(S.u.Gp[warp]);
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
// Split rows (n_i > kSplitMin): one CTA per chunk of kSplitChunk positions.
struct SplitPlan {
    const int32_t* row;      // [n_slots] row id of each slot
    const int32_t* c_begin;  // [n_slots + 1] chunk range of each slot
    const int32_t* ch_slot;  // [n_chunks]
    const int32_t* ch_start; // [n_chunks] first position of the chunk inside its row
    int n_slots;
    int n_chunks;
};

struct SplitState {  // per (slot, column) selection state and scratch
    uint32_t* P;
    uint32_t* Mk;
    int32_t* need;
    int32_t* cut;
    int32_t* done;
    uint32_t* ghist;  // [n_slots][F][256], zero between passes
    int32_t* eqc;     // [n_chunks][F]
    float* part;      // [n_chunks][F][F+1]
};

struct ChunkInfo {
    int slot;
    int64_t lo;  // absolute entry of the row start
    int n;       // row length
    int start;   // first position of the chunk
    int len;
};

__device__ __forceinline__ ChunkInfo chunk_info(const SplitPlan& sp, const Side& side, int c) {
    ChunkInfo ci;
    ci.slot = sp.ch_slot[c];
    const int64_t row = sp.row[ci.slot];
    ci.lo = side.indptr[row];
    ci.n = (int)(side.indptr[row + 1] - ci.lo);
    ci.start = sp.ch_start[c];
    ci.len = min(kSplitChunk, ci.n - ci.start);
    return ci;
}

template <int F>
__global__ void k_split_init(Side side, Params p, SplitPlan sp, SplitState st) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= sp.n_slots * F) return;
    const int slot = e / F, a = e % F;
    const int64_t row = sp.row[slot];
    const long long n = side.indptr[row + 1] - side.indptr[row];
    uint32_t P, Mk;
    int need, cut, done;
    init_column(a, p.f, row_budget(n, p), n, P, Mk, need, cut, done);
    st.P[e] = P;
    st.Mk[e] = Mk;
    st.need[e] = need;
    st.cut[e] = cut;
    st.done[e] = done;
}

template <int F>
__global__ void __launch_bounds__(kCtaThreads) k_split_hist(Side side, Params p, SplitPlan sp, SplitState st,
                                                            int pass) {
    __shared__ uint32_t hist[F][256];
    const int tid = threadIdx.x;
    const ChunkInfo ci = chunk_info(sp, side, blockIdx.x);
    for (int e = tid; e < F * 256; e += kCtaThreads) (&hist[0][0])[e] = 0u;
    __syncthreads();
    const int a_t = tid % F, k0 = tid / F;
    constexpr int kstep = kCtaThreads / F;
    const int sa = ci.slot * F + a_t;
    if (!st.done[sa]) {
        const uint32_t Pa = st.P[sa], hm = radix_before(pass);
        const int64_t e0 = ci.lo + ci.start;
        for (int k = k0; k < ci.len; k += kstep) {
            const int32_t j = side.indices[e0 + k];
            const uint32_t key = mag_key(__ldg(side.Y + (int64_t)j * p.f + a_t));
            if ((key & hm) == Pa) atomicAdd(&hist[a_t][radix_digit(key, pass)], 1u);
        }
    }
    __syncthreads();
    uint32_t* g = st.ghist + (int64_t)ci.slot * F * 256;
    for (int e = tid; e < F * 256; e += kCtaThreads) {
        const uint32_t v = (&hist[0][0])[e];
        if (v) atomicAdd(g + e, v);
    }
}

// One warp per (slot, column): pick the bin, clear the histogram row.
template <int F>
__global__ void k_split_scan(SplitPlan sp, SplitState st, int pass) {
    const int lane = threadIdx.x & 31;
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= sp.n_slots * F) return;
    if (st.done[e]) return;
    uint32_t* bins = st.ghist + (int64_t)e * 256;
    const BinPick bp = warp_pick_bin(bins, (uint32_t)st.need[e]);
#pragma unroll
    for (int q = 0; q < 8; ++q) bins[lane * 8 + q] = 0u;
    if (lane == 0) {
        st.P[e] |= (uint32_t)bp.digit << radix_shift(pass);
        st.Mk[e] = radix_after(pass);
        st.need[e] = (int)bp.newneed;
        if (bp.inbin == bp.newneed) st.done[e] = 1;
    }
}

// Keys equal to the full threshold key, per chunk and open column.
template <int F>
__global__ void __launch_bounds__(kCtaThreads) k_split_eqcount(Side side, Params p, SplitPlan sp, SplitState st) {
    __shared__ int cnt[F];
    const int tid = threadIdx.x;
    const ChunkInfo ci = chunk_info(sp, side, blockIdx.x);
    if (tid < F) cnt[tid] = 0;
    __syncthreads();
    const int a_t = tid % F, k0 = tid / F;
    constexpr int kstep = kCtaThreads / F;
    const int sa = ci.slot * F + a_t;
    if (!st.done[sa]) {
        const uint32_t T = st.P[sa];
        const int64_t e0 = ci.lo + ci.start;
        int local = 0;
        for (int k = k0; k < ci.len; k += kstep) {
            const int32_t j = side.indices[e0 + k];
            local += mag_key(__ldg(side.Y + (int64_t)j * p.f + a_t)) == T;
        }
        if (local) atomicAdd(&cnt[a_t], local);
    }
    __syncthreads();
    if (tid < F) st.eqc[(int64_t)blockIdx.x * F + tid] = cnt[tid];
}

// One warp per open (slot, column): the position cut among equal keys.
template <int F>
__global__ void k_split_cut(Side side, Params p, SplitPlan sp, SplitState st) {
    const int lane = threadIdx.x & 31;
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= sp.n_slots * F) return;
    if (st.done[e]) return;
    const int slot = e / F, a = e % F;
    const int nd = st.need[e];
    const uint32_t T = st.P[e];
    int cum = 0, cstar = -1;
    for (int c = sp.c_begin[slot]; c < sp.c_begin[slot + 1]; ++c) {
        const int q = st.eqc[(int64_t)c * F + a];
        if (cum + q >= nd) {
            cstar = c;
            break;
        }
        cum += q;
    }
    int cut = 0x7fffffff;
    if (cstar >= 0) {
        const ChunkInfo ci = chunk_info(sp, side, cstar);
        const int64_t e0 = ci.lo + ci.start;
        int seen = cum;
        for (int kb = 0; kb < ci.len; kb += 32) {
            const int k = kb + lane;
            bool eq = false;
            if (k < ci.len) eq = mag_key(__ldg(side.Y + (int64_t)side.indices[e0 + k] * p.f + a)) == T;
            unsigned b = __ballot_sync(kFull, eq);
            const int c = __popc(b);
            if (seen + c >= nd) {
                int want = nd - seen;
                while (--want > 0) b &= b - 1u;
                cut = ci.start + kb + __ffs(b);
                break;
            }
            seen += c;
        }
    }
    if (lane == 0) st.cut[e] = cut;
}

template <int F>
struct SplitGramSmem {
    float x[kSplitChunk][F];
    float r[kSplitChunk];
    int32_t idx[kSplitChunk];
    uint32_t mask[kSplitChunk];
    float Gp[kCtaWarps][F][F + 1];
};

// Masked Gram of one chunk into part[c] (or masks only when mode == 2).
template <int F>
__global__ void __launch_bounds__(kCtaThreads) k_split_gram(Side side, Params p, SplitPlan sp, SplitState st,
                                                            int mode, uint32_t* __restrict__ masks_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SplitGramSmem<F>& S = *reinterpret_cast<SplitGramSmem<F>*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = blockIdx.x;
    const ChunkInfo ci = chunk_info(sp, side, c);
    stage_tile<F>(S.x, S.r, S.idx, side, p.f, ci.lo + ci.start, ci.len);
    const int a_t = tid % F, k0 = tid / F;
    constexpr int kstep = kCtaThreads / F;
    const int sa = ci.slot * F + a_t;
    const uint32_t Pa = st.P[sa], Ma = st.Mk[sa];
    const int cuta = st.cut[sa];
    const uint32_t fmask = (F == 32) ? kFull : ((1u << F) - 1u);
    for (int kk = 0; kk < ci.len; kk += kstep) {
        const int k = kk + k0;
        const bool keep = k < ci.len && keep_rule(mag_key(S.x[k][a_t]), Pa, Ma, ci.start + k, cuta);
        const unsigned b = __ballot_sync(kFull, keep);
        if (a_t == 0 && k < ci.len) S.mask[k] = (b >> (lane & ~(F - 1))) & fmask;
    }
    __syncthreads();
    if (masks_out != nullptr)
        for (int k = tid; k < ci.len; k += kCtaThreads) masks_out[ci.lo + ci.start + k] = S.mask[k];
    if (mode == 2) return;
    GramAcc<F> g;
    g.zero();
    g.add_tile(S.x, S.mask, S.r, warp, ci.len, kCtaWarps, p.gram_mode == GRAM_SYM);
    g.store(S.Gp[warp]);
    __syncthreads();
    float* dst = st.part + (int64_t)c * F * (F + 1);
    for (int e = tid; e < F * (F + 1); e += kCtaThreads) {
        const int a = e / (F + 1), b = e % (F + 1);
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < kCtaWarps; ++q) v += S.Gp[q][a][b];
        dst[e] = v;
    }
}

// Sum the chunk Grams of each slot in chunk order, add the regulariser.
template <int F>
__global__ void __launch_bounds__(kCtaThreads) k_split_reduce(Side side, Params p, SplitPlan sp, SplitState st,
                                                              float* __restrict__ G_aug) {
    const int slot = blockIdx.x;
    const int64_t row = sp.row[slot];
    const long long n = side.indptr[row + 1] - side.indptr[row];
    const float reg = row_reg(n, p);
    const int c0 = sp.c_begin[slot], c1 = sp.c_begin[slot + 1];
    float* dst = G_aug + (int64_t)slot * F * (F + 1);
    for (int e = threadIdx.x; e < F * (F + 1); e += kCtaThreads) {
        float v = 0.f;
        for (int c = c0; c < c1; ++c) v += st.part[(int64_t)c * F * (F + 1) + e];
        const int a = e / (F + 1), b = e % (F + 1);
        if (a == b) v = (a < p.f) ? v + reg : 1.f;
        dst[e] = v;
    }
}

}  // namespace als
