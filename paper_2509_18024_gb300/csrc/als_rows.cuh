// CTA-resident rows (32 < n_i <= 1024) and split rows (n_i > 1024) of one
// Core-ALS half-sweep: CES (Algorithm 1) by exact radix select, then the
// masked Gram of Eq. (core_ui) in FP32 on CUDA cores.
#pragma once

#include <type_traits>

#include "als_device.cuh"
#include "als_tc.cuh"

namespace als {

constexpr int kCtaThreads = 256;
constexpr int kCtaWarps = kCtaThreads / 32;
constexpr int kSplitSuper = 4096;  // positions per histogram block of a split row
constexpr int kGatherBatch = 8;    // independent gathers in flight per thread
constexpr int kGramBufs = kCtaWarps / 2;  // CUDA-core Gram partial buffers per CTA
// Longest run of chunks one split-row accumulator sums before its partial is
// written (keeps the sums blocked for very long rows): 16 chunks for the
// FP32 register partials, 4 for a TMEM accumulator (the tensor cores' own
// accumulation order loses more over long runs).
__host__ __device__ constexpr int run_chunks(int eng) { return eng == 0 ? 16 : 4; }

// Gram engines: FP32 on CUDA cores (n_f <= 32), or tcgen05 in BF16, TF32,
// or split TF32 (FP32-accurate).
enum { ENG_CUDA = 0, ENG_BF16 = 1, ENG_TF32 = 2, ENG_TF32X3 = 3 };
__host__ __device__ constexpr int tc_prec(int eng) { return eng == ENG_BF16 ? TC_BF16 : (eng == ENG_TF32 ? TC_TF32 : TC_TF32X3); }

// Positions per Gram chunk of a split row, by padded width.
template <int F>
struct SplitChunk {
    static constexpr int value = F <= 32 ? 256 : (F == 64 ? 256 : 128);
};
__host__ __device__ constexpr int split_chunk(int F) { return F <= 32 ? 256 : (F == 64 ? 256 : 128); }

// Columns per histogram CTA of a split row (its shared bins: 32 x 265 words).
template <int F>
struct SplitHistCols {
    static constexpr int value = F < 32 ? F : 32;
};
// Resident CTAs per SM that k_split_gram is compiled for: one for the
// tensor-core engines (their tiles fill shared memory; without the bound the
// compiler holds them to 64 registers), three (as many as the shared memory
// allows at F = 32) or four on the CUDA cores.
__host__ __device__ constexpr int split_gram_min_blocks(int F, int eng) { return eng != 0 ? 1 : (F >= 32 ? 3 : 4); }
__host__ __device__ constexpr int split_hist_cols(int F) { return F < 32 ? F : 32; }

// Mask words per position.
template <int F>
struct MaskWords {
    static constexpr int value = (F + 31) / 32;
};

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
    // x: [*][F] row-major tile, mask: keep bits per position (F <= 32: one
    // word), r: ratings.
    __device__ __forceinline__ void add_tile(const float (*x)[xpitch(F)], const uint32_t* mask, const float* r, int k_begin,
                                             int k_end, int k_step, bool sym) {
        const int lane = threadIdx.x & 31;
        const int a0 = (lane >> 2) * TA, b0 = (lane & 3) * TB;
        for (int k = k_begin; k < k_end; k += k_step) {
            const uint32_t m = mask[k];
            float xa[TA], xb[TB];
            if constexpr (TA % 4 == 0 && TB % 4 == 0) {
                // 16-byte loads: a0 and b0 are multiples of 4.
                const float4* row = reinterpret_cast<const float4*>(x[k]);
#pragma unroll
                for (int q = 0; q < TA / 4; ++q) {
                    const float4 v = row[a0 / 4 + q];
                    xa[4 * q] = v.x;
                    xa[4 * q + 1] = v.y;
                    xa[4 * q + 2] = v.z;
                    xa[4 * q + 3] = v.w;
                }
#pragma unroll
                for (int t = 0; t < TB / 4; ++t) {
                    const float4 v = row[b0 / 4 + t];
                    xb[4 * t] = v.x;
                    xb[4 * t + 1] = v.y;
                    xb[4 * t + 2] = v.z;
                    xb[4 * t + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < TA; ++q) xa[q] = x[k][a0 + q];
#pragma unroll
                for (int t = 0; t < TB; ++t) xb[t] = x[k][b0 + t];
            }
            const uint32_t ma = m >> a0, mb = m >> b0;
#pragma unroll
            for (int q = 0; q < TA; ++q) xa[q] = ((ma >> q) & 1u) ? xa[q] : 0.f;
            if (sym) {
#pragma unroll
                for (int t = 0; t < TB; ++t) xb[t] = ((mb >> t) & 1u) ? xb[t] : 0.f;
            }
            const float rk = r[k];
#pragma unroll
            for (int q = 0; q < TA; ++q) {
                rh[q] = fmaf(xa[q], rk, rh[q]);
#pragma unroll
                for (int t = 0; t < TB; ++t) acc[q][t] = fmaf(xa[q], xb[t], acc[q][t]);
            }
        }
    }
    // Gp = this warp's partial (add: Gp += partial).
    template <bool ADD>
    __device__ __forceinline__ void store(float (*Gp)[F + 1]) const {
        const int lane = threadIdx.x & 31;
        const int a0 = (lane >> 2) * TA, b0 = (lane & 3) * TB;
#pragma unroll
        for (int q = 0; q < TA; ++q) {
#pragma unroll
            for (int t = 0; t < TB; ++t) Gp[a0 + q][b0 + t] = ADD ? Gp[a0 + q][b0 + t] + acc[q][t] : acc[q][t];
            if ((lane & 3) == 0) Gp[a0 + q][F] = ADD ? Gp[a0 + q][F] + rh[q] : rh[q];
        }
    }
};

// Stage positions [0, cn) of the slice starting at absolute entry e0. With
// f == F and a 16-byte aligned Y, each thread moves whole float4 quarters of
// rows (eight threads per 128-byte row at F = 32); else one float each, zero
// in the padding columns a >= f.
template <int F>
__device__ __forceinline__ void stage_tile(float (*x)[xpitch(F)], float* r, int32_t* idx, const Side& side, int f,
                                           int64_t e0, int cn) {
    for (int k = threadIdx.x; k < cn; k += kCtaThreads) {
        idx[k] = factor_row(side.indices[e0 + k], side.n_cols);
        r[k] = side.values[e0 + k];
    }
    __syncthreads();
    if (f == F && (reinterpret_cast<uintptr_t>(side.Y) & 15u) == 0) {
        constexpr int Q = F / 4;  // float4 per row
        constexpr int B = 4;      // independent gathers in flight per thread
        const int total = cn * Q;
        for (int g0 = threadIdx.x; g0 < total; g0 += kCtaThreads * B) {
            float4 v[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int g = g0 + u * kCtaThreads;
                v[u] = g < total ? __ldg(reinterpret_cast<const float4*>(side.Y + (int64_t)idx[g / Q] * F) + g % Q)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int g = g0 + u * kCtaThreads;
                if (g < total) reinterpret_cast<float4*>(x[g / Q])[g % Q] = v[u];
            }
        }
    } else {
        const int total = cn * F;
        for (int g0 = threadIdx.x; g0 < total; g0 += kCtaThreads * kGatherBatch) {
            float v[kGatherBatch];
#pragma unroll
            for (int u = 0; u < kGatherBatch; ++u) {
                const int e = g0 + u * kCtaThreads;
                const int k = e / F, a = e % F;
                v[u] = (e < total && a < f) ? __ldg(side.Y + (int64_t)idx[k] * f + a) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kGatherBatch; ++u) {
                const int e = g0 + u * kCtaThreads;
                if (e < total) x[e / F][e % F] = v[u];
            }
        }
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
// Keep masks of a staged tile: thread (k, g) applies the keep rules of
// columns 4g..4g+3 (state P, Mk, cut indexed by column) to one float4 of
// position k; the nibbles of one mask word meet by an OR over the (up to 8)
// neighbouring lanes of that position. pos0 = position of tile row 0 in its
// row; with gpos (the fast variant's factor-wide rule) the position of tile
// row k is gpos[k], its row index in the design factor.
template <int F>
__device__ __forceinline__ void build_masks(uint32_t (*mask)[MaskWords<F>::value], const float (*x)[xpitch(F)], int cn,
                                            int pos0, const uint32_t* P, const uint32_t* Mk, const int32_t* cut,
                                            const int32_t* gpos = nullptr) {
    static_assert(F % 4 == 0 && F / 4 <= 32, "a position's quarters sit in one warp");
    constexpr int T4 = F / 4;                  // threads per position
    constexpr int GW = T4 < 8 ? T4 : 8;        // threads per mask word
    constexpr int kstep = kCtaThreads / T4;    // positions per pass of the CTA
    const int tid = threadIdx.x;
    const int g = tid % T4, k0 = tid / T4;
    uint32_t Pc[4], Mc[4];
    int Cc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        Pc[c] = P[4 * g + c];
        Mc[c] = Mk[4 * g + c];
        Cc[c] = cut[4 * g + c];
    }
    for (int kk = 0; kk < cn; kk += kstep) {
        const int k = kk + k0;
        uint32_t nib = 0u;
        if (k < cn) {
            const float4 v = reinterpret_cast<const float4*>(x[k])[g];
            const int pos = gpos ? gpos[k] : pos0 + k;
            nib = (uint32_t)keep_rule(mag_key(v.x), Pc[0], Mc[0], pos, Cc[0]) |
                  ((uint32_t)keep_rule(mag_key(v.y), Pc[1], Mc[1], pos, Cc[1]) << 1) |
                  ((uint32_t)keep_rule(mag_key(v.z), Pc[2], Mc[2], pos, Cc[2]) << 2) |
                  ((uint32_t)keep_rule(mag_key(v.w), Pc[3], Mc[3], pos, Cc[3]) << 3);
        }
        uint32_t word = nib << (4 * (g % GW));
#pragma unroll
        for (int o = 1; o < GW; o <<= 1) word |= __shfl_xor_sync(kFull, word, o);
        if (k < cn && g % GW == 0) mask[k][g / 8] = word;
    }
}

// The CTA's Gram from the warps' register partials: they meet in kGramBufs
// shared buffers (warps w >= kGramBufs store, warps w < kGramBufs add theirs
// into buffer w), then the buffers are summed in order into out(a, c, v).
template <int F, class Out>
__device__ __forceinline__ void gram_flush(uint8_t* scratch, const GramAcc<F>& g, Out out) {
    const int tid = threadIdx.x, warp = tid >> 5;
    float (*Gp)[F][F + 1] = reinterpret_cast<float (*)[F][F + 1]>(scratch);
    if (warp >= kGramBufs) g.template store<false>(Gp[warp - kGramBufs]);
    __syncthreads();
    if (warp < kGramBufs) g.template store<true>(Gp[warp]);
    __syncthreads();
    for (int e = tid; e < F * (F + 1); e += kCtaThreads) {
        const int a = e / (F + 1), c = e % (F + 1);
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < kGramBufs; ++q) v += Gp[q][a][c];
        out(a, c, v);
    }
}

// ---------------------------------------------------------------------------
// Largest exponent of |y_a| over every row of the factor Y (n_cols x f), per
// column: tcol[a] (zeroed before the launch). The CES window of a row starts
// one above it.
template <int F>
__global__ void k_colmax(const float* __restrict__ Y, int64_t n_cols, int f, uint32_t* __restrict__ tcol) {
    __shared__ uint32_t m[F];
    for (int a = threadIdx.x; a < F; a += blockDim.x) m[a] = 0u;
    __syncthreads();
    const int64_t total = n_cols * f;
    uint32_t local = 0u;
    int la = -1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % f);
        if (a != la) {
            if (la >= 0) atomicMax(&m[la], local);
            la = a;
            local = 0u;
        }
        local = max(local, mag_key(Y[e]) >> 23);
    }
    if (la >= 0) atomicMax(&m[la], local);
    __syncthreads();
    for (int a = threadIdx.x; a < f; a += blockDim.x)
        if (m[a]) atomicMax(&tcol[a], m[a]);
}

// ---------------------------------------------------------------------------
// CES of a resident slice, one warp per quad of 4 columns (Algorithm 1 per
// column: the s largest |x_ka|, ties to the lower position), by an exact
// radix select on the magnitude keys with 64 bins per column and pass:
//   window pass: keys whose exponent E lies in [T - 16, T) go to bin
//     ((E - T + 16) << 2) | key bits 22..21 (quarter octaves). T starts one
//     above the largest exponent of the factor's column (over all its rows);
//     if the window holds fewer than `need` keys, they are all kept and the
//     window moves down (T -= 16).
//   mantissa passes: key bits 20..15, 14..9, 8..3, 2..0 of the keys equal to
//     the prefix P on the bits resolved so far (mask Mk).
// A column is done when the bin holding the need-th key is taken whole;
// keys equal to P on all 31 bits beyond that are cut by position. Bins of
// one column: 64 counts at b + 4 (b / 32) (16-byte aligned octets, read as
// two uint4 by the 8 lanes scanning that column).
constexpr int kQuadPitch = 72;
constexpr int kQuadHistWords = 4 * kQuadPitch;
__device__ __forceinline__ int mpass_shift(int m) { return m == 0 ? 15 : (m == 1 ? 9 : (m == 2 ? 3 : 0)); }
__device__ __forceinline__ uint32_t mpass_digits(int m) { return m == 3 ? 7u : 63u; }
__device__ __forceinline__ uint32_t mpass_after(int m) {
    return m == 0 ? 0xffff8000u : (m == 1 ? 0xfffffe00u : (m == 2 ? 0xfffffff8u : 0xffffffffu));
}

// Scan of the 4 columns' bins of one pass: lanes 8c..8c+7 scan column c (lane
// 8c + g holds bins 8g..8g+7) from the top bin down, clear what they read,
// and return (in every lane of the group) the packed outcome: bit 0 found,
// bit 1 the bin is taken whole, bits 2..7 the bin, bits 8..19 the keys still
// needed inside it - or, when the bins hold fewer than `need` keys, found = 0
// and bits 8..19 = need minus the keys binned.
__device__ __forceinline__ uint32_t quad_scan(uint32_t* H, bool act, uint32_t need) {
    const int lane = threadIdx.x & 31, g = lane & 7, c = lane >> 3;
    uint4* oct = reinterpret_cast<uint4*>(H + c * kQuadPitch + 8 * g + ((g >> 2) << 2));
    uint4 lo4 = make_uint4(0u, 0u, 0u, 0u), hi4 = lo4;
    if (act) {
        lo4 = oct[0];
        hi4 = oct[1];
        oct[0] = make_uint4(0u, 0u, 0u, 0u);
        oct[1] = make_uint4(0u, 0u, 0u, 0u);
    }
    const uint32_t b[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
    const uint32_t lsum = b[0] + b[1] + b[2] + b[3] + b[4] + b[5] + b[6] + b[7];
    uint32_t incl = lsum;  // keys in bins >= 8g of this column
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const uint32_t t = __shfl_down_sync(kFull, incl, o, 8);
        if (g + o < 8) incl += t;
    }
    const uint32_t above = incl - lsum;
    const bool here = act && above < need && need <= incl;
    const unsigned grp = (__ballot_sync(kFull, here) >> (8 * c)) & 0xffu;
    const uint32_t total = __shfl_sync(kFull, incl, lane & ~7);
    uint32_t out = 0u;
    if (here) {
        uint32_t cum = above;
        bool found = false;
#pragma unroll
        for (int q = 7; q >= 0; --q) {
            if (!found && cum + b[q] >= need) {
                const uint32_t nn = need - cum;
                out = 1u | ((b[q] == nn) ? 2u : 0u) | ((uint32_t)(8 * g + q) << 2) | (nn << 8);
                found = true;
            }
            if (!found) cum += b[q];
        }
    }
    out = __shfl_sync(kFull, out, (lane & ~7) + (grp ? __ffs(grp) - 1 : 0));
    if (!grp) out = (need - total) << 8;
    return out;
}

// Warp-level CES of columns 4q..4q+3 of a staged slice (n <= 4095
// positions): writes their keep rule (P, Mk, cut). H: this warp's
// kQuadHistWords bins, all zero on entry and on return.
template <int F>
__device__ __forceinline__ void quad_select(const float (*x)[xpitch(F)], int n, int f, long long s, int q, uint32_t* H,
                                            const uint32_t* __restrict__ tcol, uint32_t* P_out, uint32_t* Mk_out,
                                            int32_t* cut_out) {
    const int lane = threadIdx.x & 31;
    uint32_t P[4], Mk[4];
    int need[4], cut[4], T[4];
    bool open[4], wres[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int done;
        init_column(4 * q + c, f, s, n, P[c], Mk[c], need[c], cut[c], done);
        open[c] = !done;
        wres[c] = false;
    }
    const float4* xq = reinterpret_cast<const float4*>(&x[0][4 * q]);
    constexpr int XQ = xpitch(F) / 4;  // float4 per tile row
    // Window tops: one above the factor column's largest exponent (no key
    // of this row is above it).
#pragma unroll
    for (int c = 0; c < 4; ++c) T[c] = (int)tcol[4 * q + c] + 1;
    // Bin b (< 64) of column c sits at word c * kQuadPitch + b + ((b >> 3) & 4).
    // Window passes (at most 16 windows of 16 exponents cover all 256).
    for (int it = 0; it < 16; ++it) {
        bool act[4];
        uint32_t tlo[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            act[c] = open[c] && !wres[c];
            tlo[c] = (uint32_t)(T[c] - 16);
        }
        if (!(act[0] || act[1] || act[2] || act[3])) break;
        for (int k = lane; k < n; k += 32) {
            const float4 v = xq[k * XQ];
            const uint32_t key[4] = {mag_key(v.x), mag_key(v.y), mag_key(v.z), mag_key(v.w)};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t d = (key[c] >> 23) - tlo[c];  // window row, >= 16 outside
                const uint32_t b = (d << 2) | ((key[c] >> 21) & 3u);
                if (act[c] && d < 16u) atomicAdd(H + c * kQuadPitch + b + ((b >> 3) & 4u), 1u);
            }
        }
        __syncwarp();
        const int cs = lane >> 3;
        const uint32_t res = quad_scan(H, cs == 0 ? act[0] : cs == 1 ? act[1] : cs == 2 ? act[2] : act[3],
                                       (uint32_t)(cs == 0 ? need[0] : cs == 1 ? need[1] : cs == 2 ? need[2] : need[3]));
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t rc = __shfl_sync(kFull, res, 8 * c);
            if (!act[c]) continue;
            if (rc & 1u) {
                const uint32_t dg = (rc >> 2) & 63u;
                P[c] = ((uint32_t)(T[c] - 16 + (int)(dg >> 2)) << 23) | ((dg & 3u) << 21);
                Mk[c] = 0xffe00000u;
                need[c] = (int)(rc >> 8);
                wres[c] = true;
                if (rc & 2u) open[c] = false;
            } else {
                need[c] = (int)(rc >> 8);  // the window's keys are all kept
                T[c] -= 16;
            }
        }
        __syncwarp();
    }
    // Mantissa passes.
    for (int m = 0; m < 4; ++m) {
        if (!(open[0] || open[1] || open[2] || open[3])) break;
        const int sh = mpass_shift(m);
        const uint32_t dm = mpass_digits(m);
        for (int k = lane; k < n; k += 32) {
            const float4 v = xq[k * XQ];
            const uint32_t key[4] = {mag_key(v.x), mag_key(v.y), mag_key(v.z), mag_key(v.w)};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t b = (key[c] >> sh) & dm;
                if (open[c] && (key[c] & Mk[c]) == P[c]) atomicAdd(H + c * kQuadPitch + b + ((b >> 3) & 4u), 1u);
            }
        }
        __syncwarp();
        const int cs = lane >> 3;
        const uint32_t res = quad_scan(H, cs == 0 ? open[0] : cs == 1 ? open[1] : cs == 2 ? open[2] : open[3],
                                       (uint32_t)(cs == 0 ? need[0] : cs == 1 ? need[1] : cs == 2 ? need[2] : need[3]));
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t rc = __shfl_sync(kFull, res, 8 * c);
            if (!open[c]) continue;
            P[c] |= ((rc >> 2) & 63u) << sh;
            Mk[c] = mpass_after(m);
            need[c] = (int)(rc >> 8);
            if (rc & 2u) open[c] = false;
        }
        __syncwarp();
    }
    // Columns still open: the full key P has more copies than places left;
    // keep the lowest positions.
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (!open[c]) continue;
        int seen = 0;
        for (int kb = 0; kb < n; kb += 32) {
            const int k = kb + lane;
            unsigned bl = __ballot_sync(kFull, k < n && mag_key(x[k][4 * q + c]) == P[c]);
            const int cnt = __popc(bl);
            if (seen + cnt >= need[c]) {
                for (int want = need[c] - seen; --want > 0;) bl &= bl - 1u;
                cut[c] = kb + __ffs(bl);
                break;
            }
            seen += cnt;
        }
    }
    if (lane < 4) {
        const int c = lane;
        P_out[4 * q + c] = c == 0 ? P[0] : c == 1 ? P[1] : c == 2 ? P[2] : P[3];
        Mk_out[4 * q + c] = c == 0 ? Mk[0] : c == 1 ? Mk[1] : c == 2 ? Mk[2] : Mk[3];
        cut_out[4 * q + c] = c == 0 ? cut[0] : c == 1 ? cut[1] : c == 2 ? cut[2] : cut[3];
    }
}

// ---------------------------------------------------------------------------
// Sparse asymmetric Gram (F = 32): row a of X*^T X is the sum over the kept
// positions k of column a of x_ka X[k][:], and the rhs entry sum_k x_ka r_k,
// so only the kept positions are visited (2 s F^2 flops for a row with s
// kept per column, the count of Theorem 4). A warp owns four columns
// a = 4q .. 4q+3: it lists each column's kept positions of a staged tile
// (keep rule P, Mk, cut of the selection) and accumulates those four rows in
// registers - lane group g = lane / 8 takes row a = 4q + g, lane j = lane % 8
// its columns 4j .. 4j+3.
struct SparseAcc {
    float a0, a1, a2, a3, rh;
    __device__ __forceinline__ void zero() { a0 = a1 = a2 = a3 = rh = 0.f; }
};

// Lists the kept positions of columns 4q..4q+3 among tile rows [0, n) (tile
// row k has position pos0 + k in its row, or gpos[k] with the fast variant's
// factor-wide rule) into list (4 x lcap uint16), ORs their keep bits into
// mask[k] when mask is given, and returns the number listed for this lane's
// column.
template <int F>
__device__ __forceinline__ int sparse_list(const float (*x)[xpitch(F)], int n, int pos0, const int32_t* gpos, int q,
                                           const uint32_t* P, const uint32_t* Mk, const int32_t* cut, uint16_t* list,
                                           int lcap, uint32_t* mask) {
    static_assert(F == 32, "four columns per warp, eight lanes per row");
    const int lane = threadIdx.x & 31;
    uint32_t Pc[4], Mc[4];
    int Cc[4], cnt[4] = {0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        Pc[c] = P[4 * q + c];
        Mc[c] = Mk[4 * q + c];
        Cc[c] = cut[4 * q + c];
    }
    const unsigned below = lanemask_lt();
    for (int kb = 0; kb < n; kb += 32) {
        const int k = kb + lane;
        uint32_t nib = 0u;
        if (k < n) {
            const float4 v = reinterpret_cast<const float4*>(x[k])[q];
            const int pos = gpos ? gpos[k] : pos0 + k;
            nib = (uint32_t)keep_rule(mag_key(v.x), Pc[0], Mc[0], pos, Cc[0]) |
                  ((uint32_t)keep_rule(mag_key(v.y), Pc[1], Mc[1], pos, Cc[1]) << 1) |
                  ((uint32_t)keep_rule(mag_key(v.z), Pc[2], Mc[2], pos, Cc[2]) << 2) |
                  ((uint32_t)keep_rule(mag_key(v.w), Pc[3], Mc[3], pos, Cc[3]) << 3);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const unsigned b = __ballot_sync(kFull, (nib >> c) & 1u);
            const int at = cnt[c] + __popc(b & below);
            if (((nib >> c) & 1u) && at < lcap) list[c * lcap + at] = (uint16_t)k;
            cnt[c] += __popc(b);
        }
        if (mask != nullptr && nib) atomicOr(mask + k, nib << (4 * q));
    }
    __syncwarp();
    const int g = lane >> 3;
    return min(g == 0 ? cnt[0] : g == 1 ? cnt[1] : g == 2 ? cnt[2] : cnt[3], lcap);
}

// Adds the listed positions of this lane's column to acc.
template <int F>
__device__ __forceinline__ void sparse_accum(const float (*x)[xpitch(F)], const float* r, int q, const uint16_t* list,
                                             int lcap, int na, SparseAcc& acc) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 3, j = lane & 7, a = 4 * q + g;
    const uint16_t* la = list + g * lcap;
    for (int t = 0; t < na; ++t) {
        const int k = la[t];
        const float xa = x[k][a];
        const float4 xb = reinterpret_cast<const float4*>(x[k])[j];
        acc.a0 = fmaf(xa, xb.x, acc.a0);
        acc.a1 = fmaf(xa, xb.y, acc.a1);
        acc.a2 = fmaf(xa, xb.z, acc.a2);
        acc.a3 = fmaf(xa, xb.w, acc.a3);
        acc.rh = fmaf(xa, r[k], acc.rh);
    }
}

// Stores the warp's four rows of [G | b] to dst (F x (F + 1)); with `diag`
// the regulariser goes on the diagonal and padding rows (a >= f) become
// identity rows, else the raw sums are stored (a split row's partial).
template <int F>
__device__ __forceinline__ void sparse_store(const SparseAcc& acc, int q, int f, float reg, bool diag, float* dst) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 3, j = lane & 7, a = 4 * q + g;
    float* row = dst + a * (F + 1);
    const float v[4] = {acc.a0, acc.a1, acc.a2, acc.a3};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int c = 4 * j + e;
        row[c] = (diag && a == c) ? ((a < f) ? v[e] + reg : 1.f) : v[e];
    }
    if (j == 0) row[F] = acc.rh;
}

// ---------------------------------------------------------------------------
// CTA per row, slice resident in shared memory.
// Bytes of the two tensor-core tile buffers of an engine (16 for CUDA cores).
template <int F, int ENG>
struct TileBytes {
    static constexpr int value = ENG == ENG_CUDA ? 16 : 2 * TcCfg<F, tc_prec(ENG)>::TILE_BYTES;
};

// Shared memory of k_cta_rows, in bytes from the (1024-byte aligned) base:
// a fixed part - tensor-core tiles, per-warp selection bins, barriers, the
// keep rules of the F columns - then the staged slice [x | r | idx | mask],
// sized for the launch's capacity (its longest row). The CUDA-core Gram's
// per-warp partials reuse the x area once the tile has been consumed.
template <int F, int ENG>
struct CtaLayout {
    static constexpr int W = MaskWords<F>::value;
    static constexpr size_t HIST_BYTES = (size_t)kCtaWarps * kQuadHistWords * 4;
    static constexpr size_t GRAM_BYTES = ENG == ENG_CUDA ? (size_t)kGramBufs * F * (F + 1) * 4 : 0;
    static constexpr size_t up16(size_t b) { return (b + 15) / 16 * 16; }
    static constexpr size_t tiles = 0;
    static constexpr size_t u = up16(TileBytes<F, ENG>::value);
    static constexpr size_t bars = u + HIST_BYTES;
    static constexpr size_t tmem_slot = bars + 2 * sizeof(uint64_t);
    static constexpr size_t row = tmem_slot + 16;  // the row's budget s_i (8 bytes) and regulariser (4)
    static constexpr size_t P = row + 16;
    static constexpr size_t Mk = P + (size_t)F * 4;
    static constexpr size_t cut = Mk + (size_t)F * 4;
    static constexpr size_t x = up16(cut + (size_t)F * 4);
    __host__ __device__ static constexpr size_t x_bytes(int cap) {
        return (size_t)cap * xpitch(F) * 4 > GRAM_BYTES ? (size_t)cap * xpitch(F) * 4 : GRAM_BYTES;
    }
    __host__ __device__ static constexpr size_t r(int cap) { return x + x_bytes(cap); }
    __host__ __device__ static constexpr size_t idx(int cap) { return r(cap) + (size_t)cap * 4; }
    __host__ __device__ static constexpr size_t mask(int cap) { return idx(cap) + (size_t)cap * 4; }
    // Kept-position lists of the sparse asymmetric Gram (CUDA cores, F = 32):
    // per warp 4 columns x cap / 4 positions (uint16).
    static constexpr bool SPARSE = ENG == ENG_CUDA && F == 32;
    __host__ __device__ static constexpr int list_cap(int cap) { return cap / 4; }
    __host__ __device__ static constexpr size_t list(int cap) { return up16(mask(cap) + (size_t)cap * W * 4); }
    __host__ __device__ static constexpr size_t bytes(int cap) {
        return up16(list(cap) + (SPARSE ? (size_t)kCtaWarps * 4 * list_cap(cap) * 2 : 0));
    }
};

// mode 0/1: write the augmented system of list entry w to G_aug[w]; mode 2:
// masks only. Every listed row has at most `cap` positions (the capacity the
// shared memory was sized for). CTAs loop over list entries w = blockIdx.x +
// k gridDim.x; with a tensor-core engine the grid is persistent, TMEM and
// tiles are set up once per CTA, and each row's accumulator is read back
// after the next row has been staged and selected (its MMAs run meanwhile).
template <int F, int ENG>
__global__ void __launch_bounds__(kCtaThreads, ENG == ENG_CUDA ? 4 : 2) k_cta_rows(Side side, Params p, const int32_t* __restrict__ rows,
                                                          int n_list, int cap, int mode, float* __restrict__ G_aug,
                                                          uint32_t* __restrict__ masks_out,
                                                          const uint32_t* __restrict__ tcol) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using L = CtaLayout<F, ENG>;
    constexpr int W = L::W;
    uint8_t* const s_tiles = smem_raw + L::tiles;
    uint8_t* const s_u = smem_raw + L::u;
    uint64_t* const s_bars = reinterpret_cast<uint64_t*>(smem_raw + L::bars);
    uint32_t* const s_tmem = reinterpret_cast<uint32_t*>(smem_raw + L::tmem_slot);
    long long* const s_budget = reinterpret_cast<long long*>(smem_raw + L::row);
    float* const s_reg = reinterpret_cast<float*>(smem_raw + L::row + 8);
    uint32_t* const s_P = reinterpret_cast<uint32_t*>(smem_raw + L::P);
    uint32_t* const s_Mk = reinterpret_cast<uint32_t*>(smem_raw + L::Mk);
    int32_t* const s_cut = reinterpret_cast<int32_t*>(smem_raw + L::cut);
    float (*const s_x)[xpitch(F)] = reinterpret_cast<float (*)[xpitch(F)]>(smem_raw + L::x);
    float* const s_r = reinterpret_cast<float*>(smem_raw + L::r(cap));
    int32_t* const s_idx = reinterpret_cast<int32_t*>(smem_raw + L::idx(cap));
    uint32_t (*const s_mask)[W] = reinterpret_cast<uint32_t (*)[W]>(smem_raw + L::mask(cap));
    uint16_t* const s_list = reinterpret_cast<uint16_t*>(smem_raw + L::list(cap));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int f = p.f;
    constexpr bool TC = ENG != ENG_CUDA;
    constexpr int PREC = TC ? tc_prec(ENG) : 0;
    const bool sym = p.gram_mode == GRAM_SYM;
    TcPipe P;
    if constexpr (TC) {
        if (mode != 2 && blockIdx.x < n_list) tc_pipe_setup<F, PREC>(s_tiles, s_bars, s_tmem, P, p.err);
    }
    // This warp's selection bins: zeroed once, every selection leaves them zero.
    uint32_t* const H = reinterpret_cast<uint32_t*>(s_u) + warp * kQuadHistWords;
    for (int e = lane; e < kQuadHistWords / 4; e += 32) reinterpret_cast<uint4*>(H)[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    // Fast variant: every row applies the factor-wide keep rule.
    const bool factor_rule = p.gP != nullptr;
    if (factor_rule)
        for (int a = tid; a < F; a += kCtaThreads) {
            s_P[a] = p.gP[a];
            s_Mk[a] = p.gMk[a];
            s_cut[a] = p.gcut[a];
        }
    int prev_w = -1, prev_n = 0, prev_acc = 0, iter = 0;
    float prev_reg = 0.f;
    auto finish_prev = [&]() {
        if constexpr (TC) {
            if (prev_w < 0) return;
            float* dst = G_aug + (int64_t)prev_w * F * (F + 1);
            const float reg = prev_reg;
            // The selection bins are free here (every warp has selected this
            // row's columns): they carry the transpose, then are cleared.
            static_assert(L::HIST_BYTES >= kTcStoreBufFloats * 4, "transpose buffer in the bins");
            tc_pipe_finish<F, PREC>(
                P, s_bars, prev_acc, prev_n == 0,
                [&](int a, int c, float v) {
                    if (a == c) v = (a < f) ? v + reg : 1.f;
                    dst[a * (F + 1) + c] = v;
                },
                reinterpret_cast<float*>(s_u));
            __syncthreads();
            for (int e = tid; e < (int)(L::HIST_BYTES / 16); e += kCtaThreads)
                reinterpret_cast<uint4*>(s_u)[e] = make_uint4(0u, 0u, 0u, 0u);
            prev_w = -1;
        }
    };
    for (int w = blockIdx.x; w < n_list; w += gridDim.x, ++iter) {
    __syncthreads();
    const int64_t i = rows[w];
    const int64_t lo = side.indptr[i];
    const int n = min((int)(side.indptr[i + 1] - lo), cap);  // the plan's bound on this launch's rows
    // The budget and regulariser take FP64 steps (a slow pipe here): one
    // thread evaluates them; stage_tile's barrier publishes them.
    if (tid == 0) {
        *s_budget = row_budget(n, p);
        *s_reg = row_reg(n, p);
    }
    // Sparse asymmetric Gram (CUDA cores, F = 32, Algorithm 2's exact budget
    // s per column, s <= cap / 4): the warp that selected columns 4w..4w+3
    // lists their kept positions and assembles rows 4w..4w+3 of X*^T X, with
    // no CTA barrier between selection and Gram. The choice depends on the
    // row's budget only, so every thread takes the same branch. Its mask
    // words start at zero (the warps OR their columns' bits into them).
    if constexpr (L::SPARSE)
        if (masks_out != nullptr)
            for (int e = tid; e < n * W; e += kCtaThreads) (&s_mask[0][0])[e] = 0u;
    stage_tile<F>(s_x, s_r, s_idx, side, f, lo, n);
    const long long s = *s_budget;
    const float reg = *s_reg;
    bool sparse = false;
    if constexpr (L::SPARSE)
        sparse = mode != 2 && p.gram_mode == GRAM_ASYM && !factor_rule && s <= (long long)L::list_cap(cap);
    // CES: warp w selects the column quads w, w + 8, ... on its own bins.
    if (!factor_rule)
        for (int q = warp; q < F / 4; q += kCtaWarps) quad_select<F>(s_x, n, f, s, q, H, tcol, s_P, s_Mk, s_cut);
    if constexpr (L::SPARSE) {
        if (sparse) {
            __syncwarp();
            uint16_t* lw = s_list + warp * 4 * L::list_cap(cap);
            const int na = sparse_list<F>(s_x, n, 0, nullptr, warp, s_P, s_Mk, s_cut, lw, L::list_cap(cap),
                                          masks_out != nullptr ? &s_mask[0][0] : nullptr);
            SparseAcc acc;
            acc.zero();
            sparse_accum<F>(s_x, s_r, warp, lw, L::list_cap(cap), na, acc);
            sparse_store<F>(acc, warp, f, reg, true, G_aug + (int64_t)w * F * (F + 1));
            if (masks_out != nullptr) {
                __syncthreads();
                for (int e = tid; e < n * W; e += kCtaThreads) masks_out[lo * W + e] = (&s_mask[0][0])[e];
            }
            continue;
        }
    }
    __syncthreads();
    build_masks<F>(s_mask, s_x, n, 0, s_P, s_Mk, s_cut, factor_rule ? s_idx : nullptr);
    __syncthreads();
    if (masks_out != nullptr)
        for (int e = tid; e < n * W; e += kCtaThreads) masks_out[lo * W + e] = (&s_mask[0][0])[e];
    if (mode == 2) continue;
    if constexpr (TC) {
        finish_prev();
        tc_pipe_row<F, PREC, W>(P, s_tiles, s_bars, s_x, s_mask, s_r, n, sym, iter & 1);
        prev_w = w;
        prev_n = n;
        prev_reg = reg;
        prev_acc = iter & 1;
    } else {
        float* dst = G_aug + (int64_t)w * F * (F + 1);
        GramAcc<F> g;
        g.zero();
        g.add_tile(s_x, &s_mask[0][0], s_r, warp, n, kCtaWarps, sym);
        __syncthreads();  // the partials overwrite the x area
        gram_flush<F>(smem_raw + L::x, g, [&](int a, int c, float v) {
            if (a == c) v = (a < f) ? v + reg : 1.f;
            dst[a * (F + 1) + c] = v;
        });
    }
    }  // rows of this CTA
    if constexpr (TC) {
        if (mode != 2 && blockIdx.x < n_list) {
            finish_prev();
            tc_pipe_teardown<F, PREC>(P, s_bars);
        }
    }
}

// ---------------------------------------------------------------------------
// Split rows (longer than the largest resident bucket): Gram chunks of
// SplitChunk<F> positions, histogram blocks of kSplitSuper positions.
struct SplitPlan {
    const int32_t* row;      // [n_slots] row id of each slot
    const int32_t* c_begin;  // [n_slots + 1] chunk range of each slot
    const int32_t* ch_slot;  // [n_chunks]
    const int32_t* ch_start; // [n_chunks] first position of the chunk inside its row
    const int32_t* sc_slot;  // [n_super] histogram blocks: slot
    const int32_t* sc_start; // [n_super] first position
    int n_slots;
    int n_chunks;
    int n_super;
};

struct SplitState {  // per (slot, column) selection state and scratch
    uint32_t* P;
    uint32_t* Mk;
    int32_t* need;
    int32_t* cut;
    int32_t* done;
    uint32_t* ghist;  // [n_slots][F][256], zero between passes
    int32_t* arrive;  // [n_slots] super-chunks done with the current pass, zero between passes
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

template <int F>
__device__ __forceinline__ ChunkInfo chunk_info(const SplitPlan& sp, const Side& side, int c) {
    ChunkInfo ci;
    ci.slot = sp.ch_slot[c];
    const int64_t row = sp.row[ci.slot];
    ci.lo = side.indptr[row];
    ci.n = (int)(side.indptr[row + 1] - ci.lo);
    ci.start = sp.ch_start[c];
    ci.len = min(SplitChunk<F>::value, ci.n - ci.start);
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
__global__ void __launch_bounds__(kCtaThreads, 6) k_split_hist(Side side, Params p, SplitPlan sp, SplitState st,
                                                            int pass) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint32_t (*hist)[kHistRow] = reinterpret_cast<uint32_t (*)[kHistRow]>(smem_raw);
    constexpr int CG = SplitHistCols<F>::value;  // columns of this CTA's group
    constexpr int NG = F / CG;
    const int tid = threadIdx.x;
    const int sc = blockIdx.x / NG, grp = blockIdx.x % NG;
    const int slot = sp.sc_slot[sc];
    const int64_t row = sp.row[slot];
    const int64_t lo = side.indptr[row];
    const int n = (int)(side.indptr[row + 1] - lo);
    const int start = sp.sc_start[sc];
    const int len = min(kSplitSuper, n - start);
    for (int e = tid; e < CG * kHistRow; e += kCtaThreads) (&hist[0][0])[e] = 0u;
    __syncthreads();
    // Thread (k, q) covers columns 4q..4q+3 of its group of positions k0,
    // k0 + kstep, ...: one index load and one float4 gather (f == F, aligned
    // Y) per position.
    constexpr int T4 = CG / 4;
    constexpr int kstep = kCtaThreads / T4;
    const int q = tid % T4, k0 = tid / T4;
    const int col0 = grp * CG + 4 * q;  // first column of this thread
    const int sa = slot * F + col0;
    bool open[4];
    uint32_t Pc[4];
    bool any = false;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        open[c] = !st.done[sa + c];
        Pc[c] = st.P[sa + c];
        any |= open[c];
    }
    if (any) {
        const uint32_t hm = radix_before(pass);
        const int64_t e0 = lo + start;
        const int f = p.f;
        const bool vec = f == F && (reinterpret_cast<uintptr_t>(side.Y) & 15u) == 0;
        constexpr int B = 4;
        for (int kb = k0; kb < len; kb += kstep * B) {
            int32_t j[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int k = kb + u * kstep;
                j[u] = k < len ? factor_row(side.indices[e0 + k], side.n_cols) : -1;
            }
            float4 v[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                if (j[u] < 0) {
                    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                } else if (vec) {
                    v[u] = __ldg(reinterpret_cast<const float4*>(side.Y + (int64_t)j[u] * F + col0));
                } else {
                    const float* y = side.Y + (int64_t)j[u] * f;
                    const int a = col0;
                    v[u] = make_float4(a < f ? __ldg(y + a) : 0.f, a + 1 < f ? __ldg(y + a + 1) : 0.f,
                                       a + 2 < f ? __ldg(y + a + 2) : 0.f, a + 3 < f ? __ldg(y + a + 3) : 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                if (j[u] < 0) continue;
                const uint32_t key[4] = {mag_key(v[u].x), mag_key(v[u].y), mag_key(v[u].z), mag_key(v[u].w)};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (open[c] && (key[c] & hm) == Pc[c])
                        atomicAdd(&hist[4 * q + c][hist_slot(radix_digit(key[c], pass))], 1u);
                }
            }
        }
    }
    __syncthreads();
    uint32_t* g = st.ghist + ((int64_t)slot * F + grp * CG) * 256;
    for (int e = tid; e < CG * 256; e += kCtaThreads) {
        const uint32_t v = hist[e >> 8][hist_slot(e & 255)];
        if (v) atomicAdd(g + e, v);
    }
    // The super-chunk that finishes the slot's pass last picks the bins of
    // its open columns (an arrival count; nothing waits). Fences order this
    // CTA's histogram adds before its arrival, and the arrivals before the
    // last CTA's reads.
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(st.arrive + slot, 1) == NG * ((n + kSplitSuper - 1) / kSplitSuper) - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int warp = tid >> 5, lane = tid & 31;
    for (int a = warp; a < F; a += kCtaWarps) {
        const int e = slot * F + a;
        if (st.done[e]) continue;
        const BinPick bp = warp_pick_bin(st.ghist + (int64_t)e * 256, (uint32_t)st.need[e]);
        if (lane == 0) {
            st.P[e] |= (uint32_t)bp.digit << radix_shift(pass);
            st.Mk[e] = radix_after(pass);
            st.need[e] = (int)bp.newneed;
            if (bp.inbin == bp.newneed) st.done[e] = 1;
        }
    }
    if (tid == 0) st.arrive[slot] = 0;
}

// Keys equal to the full threshold key, per chunk and open column.
template <int F>
__global__ void __launch_bounds__(kCtaThreads) k_split_eqcount(Side side, Params p, SplitPlan sp, SplitState st) {
    __shared__ int cnt[F];
    const int tid = threadIdx.x;
    const ChunkInfo ci = chunk_info<F>(sp, side, blockIdx.x);
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
            const int32_t j = factor_row(side.indices[e0 + k], side.n_cols);
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
        const ChunkInfo ci = chunk_info<F>(sp, side, cstar);
        const int64_t e0 = ci.lo + ci.start;
        int seen = cum;
        for (int kb = 0; kb < ci.len; kb += 32) {
            const int k = kb + lane;
            bool eq = false;
            if (k < ci.len)
                eq = mag_key(__ldg(side.Y + (int64_t)factor_row(side.indices[e0 + k], side.n_cols) * p.f + a)) == T;
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

template <int F, int ENG>
struct SplitGramSmem {
    static constexpr int CH = SplitChunk<F>::value;
    static constexpr int W = MaskWords<F>::value;
    float x[CH][xpitch(F)];
    float r[CH];
    int32_t idx[CH];
    uint32_t mask[CH][W];
    // CUDA cores: the warps' Gram partials; tensor cores: the transpose
    // buffer of the accumulator read-back.
    __align__(1024) uint8_t u[ENG == ENG_CUDA ? kGramBufs * F * (F + 1) * 4 : kTcStoreBufFloats * 4];
    __align__(1024) uint8_t tiles[TileBytes<F, ENG>::value];
    uint64_t bars[2];
    uint32_t tmem_slot;
};

// Masked Gram of split chunks (or masks only when mode == 2). CTA b takes the
// contiguous chunks [b per, (b+1) per) and keeps one accumulator across
// consecutive chunks of one row (register partials on CUDA cores, a TMEM
// accumulator on tensor cores), for at most run_chunks(ENG) chunks; the run's
// Gram goes to part[first chunk of the run]. A run starts at a range start, a
// row start, or run_chunks(ENG) chunks after the previous run start. With tensor
// cores a run's accumulator is read back while the next run's first chunk is
// staged and its MMAs run.
template <int F, int ENG>
__global__ void __launch_bounds__(kCtaThreads, split_gram_min_blocks(F, ENG)) k_split_gram(Side side, Params p, SplitPlan sp, SplitState st,
                                                            int mode, uint32_t* __restrict__ masks_out, int per) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using Smem = SplitGramSmem<F, ENG>;
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    constexpr int W = Smem::W;
    constexpr bool TC = ENG != ENG_CUDA;
    constexpr int PREC = TC ? tc_prec(ENG) : 0;
    const int tid = threadIdx.x;
    const bool sym = p.gram_mode == GRAM_SYM;
    TcPipe P;
    if constexpr (TC) {
        if (mode != 2 && blockIdx.x < sp.n_chunks) tc_pipe_setup<F, PREC>(S.tiles, S.bars, &S.tmem_slot, P, p.err);
    }
    int prev_c = -1, prev_acc = 0, prev_len = 0, runs = 0;
    auto finish_prev = [&]() {
        if constexpr (TC) {
            if (prev_c < 0) return;
            float* dst = st.part + (int64_t)prev_c * F * (F + 1);
            tc_pipe_finish<F, PREC>(
                P, S.bars, prev_acc, prev_len == 0, [&](int a, int cc, float v) { dst[a * (F + 1) + cc] = v; },
                reinterpret_cast<float*>(S.u));
            prev_c = -1;
        }
    };
    const int c_first = blockIdx.x * per;
    const int c_end = min(c_first + per, sp.n_chunks);
    GramAcc<F> acc;  // CUDA cores: the current run's warp partials
    if constexpr (!TC) acc.zero();
    int run_start = c_first;
    for (int c = c_first; c < c_end; ++c) {
        __syncthreads();
        const ChunkInfo ci = chunk_info<F>(sp, side, c);
        stage_tile<F>(S.x, S.r, S.idx, side, p.f, ci.lo + ci.start, ci.len);
        if (p.gP != nullptr)  // fast variant: the factor-wide keep rule
            build_masks<F>(S.mask, S.x, ci.len, ci.start, p.gP, p.gMk, p.gcut, S.idx);
        else
            build_masks<F>(S.mask, S.x, ci.len, ci.start, st.P + ci.slot * F, st.Mk + ci.slot * F,
                           st.cut + ci.slot * F);
        __syncthreads();
        if (masks_out != nullptr)
            for (int e = tid; e < ci.len * W; e += kCtaThreads)
                masks_out[(ci.lo + ci.start) * W + e] = (&S.mask[0][0])[e];
        if (mode == 2) continue;
        if constexpr (TC) {
            const bool fresh = c == c_first || sp.ch_slot[c - 1] != ci.slot || c - run_start == run_chunks(ENG);
            if (fresh) {
                finish_prev();  // the previous run (its MMAs overlap this chunk's staging)
                run_start = c;
                ++runs;
            }
            tc_pipe_row<F, PREC, W>(P, S.tiles, S.bars, S.x, S.mask, S.r, ci.len, sym, runs & 1, fresh);
            prev_c = run_start;
            prev_acc = runs & 1;
            prev_len = ci.len;
        } else {
            acc.add_tile(S.x, &S.mask[0][0], S.r, tid >> 5, ci.len, kCtaWarps, sym);
            if (c + 1 == c_end || sp.ch_slot[c + 1] != ci.slot || c + 1 - run_start == run_chunks(ENG)) {
                float* dst = st.part + (int64_t)run_start * F * (F + 1);
                gram_flush<F>(S.u, acc, [&](int a, int cc, float v) { dst[a * (F + 1) + cc] = v; });
                acc.zero();
                run_start = c + 1;
            }
        }
    }
    if constexpr (TC) {
        if (mode != 2 && blockIdx.x < sp.n_chunks) {
            finish_prev();
            tc_pipe_teardown<F, PREC>(P, S.bars);
        }
    }
}

// Sum the partial Grams of each slot in chunk order, add the regulariser.
// A chunk holds a partial when it starts a run (see k_split_gram): the row's
// first chunk, then from each run start the next multiple of `per` (the
// chunk range of a CTA) or `run` chunks on, whichever comes first.
template <int F>
__global__ void __launch_bounds__(kCtaThreads) k_split_reduce(Side side, Params p, SplitPlan sp, SplitState st,
                                                              float* __restrict__ G_aug, int per, int run) {
    const int slot = blockIdx.x;
    const int64_t row = sp.row[slot];
    const long long n = side.indptr[row + 1] - side.indptr[row];
    const float reg = row_reg(n, p);
    const int c0 = sp.c_begin[slot], c1 = sp.c_begin[slot + 1];
    const int rb0 = (c0 / per + 1) * per;
    float* dst = G_aug + (int64_t)slot * F * (F + 1);
    for (int e = threadIdx.x; e < F * (F + 1); e += kCtaThreads) {
        float v = 0.f;
        // Run starts: inside each CTA range an arithmetic progression of step
        // `run` from the row's (or the range's) first chunk; four at a time.
        const float* pe = st.part + e;
        constexpr int64_t G = (int64_t)F * (F + 1);
        for (int c = c0, bound = rb0; c < c1; bound += per) {
            const int end = min(bound, c1);
            for (; c + 3 * run < end; c += 4 * run) {
                const float a0 = pe[c * G], a1 = pe[(c + run) * G], a2 = pe[(c + 2 * run) * G],
                            a3 = pe[(c + 3 * run) * G];
                v += ((a0 + a1) + a2) + a3;
            }
            for (; c < end; c += run) v += pe[c * G];
            c = end;
        }
        const int a = e / (F + 1), b = e % (F + 1);
        if (a == b) v = (a < p.f) ? v + reg : 1.f;
        dst[e] = v;
    }
}

}  // namespace als
