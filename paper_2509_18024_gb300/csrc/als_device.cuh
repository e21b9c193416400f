// Device-side building blocks of the core-elements ALS half-sweep (sm_103a).
//
// Notation follows the paper: a row i of one side has n_i observations I_i;
// its design slice is X = Y[I_i] (n_i x n_f) with Y the other side's factor;
// CES (Algorithm 1) keeps, in each column a of X, the s_i = floor(n_i r)
// entries of largest |x_ka| (ties: lower position k first); Eq. (core_ui)
// solves (X*^T X + lambda n_i E) x_i = X*^T r_i.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace als {

enum { GRAM_ASYM = 0, GRAM_SYM = 1, GRAM_FULL = 2 };
enum { REG_WEIGHTED = 0, REG_PLAIN = 1 };
enum { FLAG_RATIO = 1, FLAG_SINGULAR = 2, FLAG_FP64 = 4 };

constexpr unsigned kFull = 0xffffffffu;

// Row pitch (floats) of a staged slice tile: n_f plus one float4, so that a
// warp reading one 4-column quad of 32 consecutive positions as float4 hits
// all 32 banks once per quarter-warp (a pitch of n_f alone would put every
// position of a quad in the same four banks).
__host__ __device__ constexpr int xpitch(int F) { return F + 4; }

struct Params {
    int f;               // rank n_f (<= F, the compile-time padded width)
    float lambda;
    double budget;       // r
    long long min_keep;  // 0 = off
    long long fixed_keep;  // 0 = the rate rule; > 0: fixed subsample size
    int reg_mode;
    int gram_mode;
    float ratio_max;     // pivot-ratio flag threshold
    unsigned* err;       // sticky device error word (bit 0: a bounded wait ran out), or null
    // Fast variant (CES once on the whole design factor Y): the keep rule of
    // each column over Y's rows, positions being Y's row indices. Null: the
    // per-slice CES of Algorithm 2.
    const uint32_t* gP;
    const uint32_t* gMk;
    const int32_t* gcut;
};

struct Side {
    const int64_t* indptr;
    const int32_t* indices;
    const float* values;
    const float* Y;      // other side's factor, n_cols x f
    int64_t n_rows;
    int64_t n_cols;
};

// Report counters of one half-sweep (device resident).
struct Counters {
    unsigned long long flagged;
    unsigned long long singular;
    unsigned int max_ratio_bits;  // float bits of the largest finite pivot ratio
    unsigned int error;           // device-side error word (0 = none)
    unsigned long long fp64_rows; // rows re-solved in FP64
    unsigned int fb_count;        // entries in the FP64 fallback list
    unsigned int pad;
};

// Rows whose FP32 solve was flagged are appended here for the FP64 redo
// (rows == nullptr: fallback off).
struct Fallback {
    int32_t* rows;
    unsigned int* count;
};

// A column index of the rating structure as a row of the other side's factor
// (n_cols rows): indices outside [0, n_cols) - possible only when validated
// buffers were refilled in place, which the next report then flags - are
// clamped, so that no gather reads outside the factor.
__device__ __forceinline__ int32_t factor_row(int32_t j, int64_t n_cols) {
    return (uint32_t)j < (uint64_t)n_cols ? j : (j < 0 ? 0 : (int32_t)(n_cols - 1));
}

// |x| as an order-preserving unsigned key: for finite floats the unsigned
// order of the sign-cleared bit pattern is the order of |x|; -0 and +0 tie.
__device__ __forceinline__ uint32_t mag_key(float x) { return __float_as_uint(x) & 0x7fffffffu; }

// s_i = floor(n_i * r) in IEEE double (the same expression as the oracle),
// or min(n_i, fixed_keep) for a fixed subsample size; optionally raised to
// min_keep; n_i for the full update.
__device__ __forceinline__ long long row_budget(long long n, const Params& p) {
    if (p.gram_mode == GRAM_FULL) return n;
    long long s;
    if (p.fixed_keep > 0) {
        s = p.fixed_keep < n ? p.fixed_keep : n;
    } else {
        double prod = (double)n * p.budget;
        s = (long long)floor(prod);
    }
    if (s > n) s = n;
    if (s < 0) s = 0;
    if (p.min_keep > 0 && s < p.min_keep) s = p.min_keep < n ? p.min_keep : n;
    return s;
}

// Regulariser added on the diagonal: lambda n_i (weighted) or lambda.
__device__ __forceinline__ float row_reg(long long n, const Params& p) {
    return p.reg_mode == REG_PLAIN ? p.lambda : (float)((double)p.lambda * (double)n);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ unsigned lanemask_gt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_gt;" : "=r"(m));
    return m;
}

// Warp-wide CES on one column of a slice with n <= 32 elements, element k
// held by lane k. Returns the keep mask (bit k). Exact: the s largest keys,
// equal keys taken from the lowest lanes. When s <= n - s it extracts maxima
// s times at most; otherwise it removes the n - s smallest (equal keys leave
// from the highest lanes), which yields the same set.
__device__ __forceinline__ unsigned warp_ces_column(uint32_t key, int n, int s) {
    const int lane = threadIdx.x & 31;
    const unsigned valid = (n >= 32) ? kFull : ((1u << n) - 1u);
    if (s <= 0) return 0u;
    if (s >= n) return valid;
    if (2 * s <= n) {
        // key + 1 never overflows (keys <= 0x7fffffff); removed lanes hold 0.
        uint32_t k1 = (lane < n) ? key + 1u : 0u;
        unsigned sel = 0u;
        int need = s;
        // Each round takes at least one of <= 32 elements: at most 32 rounds.
        for (int round = 0; need > 0 && round < 32; ++round) {
            uint32_t m = __reduce_max_sync(kFull, k1);
            unsigned eq = __ballot_sync(kFull, k1 == m);
            unsigned take;
            if (__popc(eq) <= need) {
                take = eq;
            } else {
                bool mine = ((eq >> lane) & 1u) && (__popc(eq & lanemask_lt()) < need);
                take = __ballot_sync(kFull, mine);
            }
            sel |= take;
            need -= __popc(take);
            if ((take >> lane) & 1u) k1 = 0u;
        }
        return sel;
    } else {
        uint32_t k2 = (lane < n) ? key : 0xffffffffu;
        unsigned excl = 0u;
        int need = n - s;
        // Each round takes at least one of <= 32 elements: at most 32 rounds.
        for (int round = 0; need > 0 && round < 32; ++round) {
            uint32_t m = __reduce_min_sync(kFull, k2);
            unsigned eq = __ballot_sync(kFull, k2 == m) & valid;
            unsigned take;
            if (__popc(eq) <= need) {
                take = eq;
            } else {
                bool mine = ((eq >> lane) & 1u) && (__popc(eq & lanemask_gt()) < need);
                take = __ballot_sync(kFull, mine);
            }
            excl |= take;
            need -= __popc(take);
            if ((take >> lane) & 1u) k2 = 0xffffffffu;
        }
        return valid & ~excl;
    }
}

// Warp-cooperative solve of one F x F system held row-per-lane: lane i < F
// holds row i of A in v[0..F-1] and b_i in rhs. Gaussian elimination; with
// `pivot` true the pivot of step k is the remaining row with the largest
// |a_ik| (lowest lane on ties) - partial pivoting without moving data - else
// the diagonal (the symmetric positive definite modes, where the pivots are
// the squared Cholesky diagonal L_kk^2). Rows a >= f are padding (identity).
// Returns the solution component of this lane's column (lane < F) through
// x_lane; flags and the pivot ratio max/min over the first f pivots.
template <int F>
__device__ __forceinline__ void warp_solve(float (&v)[F], float rhs, int f, bool pivot, float ratio_max,
                                           float& x_lane, int& flags, float& ratio) {
    const int lane = threadIdx.x & 31;
    bool active = lane < F;
    int ord = -1;      // elimination step at which this lane's row was the pivot
    float upiv = 1.f;  // that pivot (the diagonal of the upper factor)
    float pmax = 0.f, pmin = __int_as_float(0x7f800000);
    bool singular = false;
#pragma unroll
    for (int k = 0; k < F; ++k) {
        int bl;
        if (pivot) {
            // Largest |a_ik| over the remaining rows, lowest lane on ties:
            // the bit patterns of non-negative floats sort like their values
            // (+1 keeps inactive lanes, 0, below every candidate).
            const uint32_t key = active ? (__float_as_uint(fabsf(v[k])) + 1u) : 0u;
            const uint32_t best = __reduce_max_sync(kFull, key);
            bl = __ffs(__ballot_sync(kFull, key == best)) - 1;
        } else {
            bl = k;
        }
        float pv = __shfl_sync(kFull, v[k], bl);
        float apv = pivot ? fabsf(pv) : pv;
        if (k < f) {
            if (!(apv > 0.f)) singular = true;
            pmax = fmaxf(pmax, apv);
            pmin = fminf(pmin, apv);
        }
        float l = (active && lane != bl && pv != 0.f) ? v[k] / pv : 0.f;
#pragma unroll
        for (int j = k + 1; j < F; ++j) {
            float pj = __shfl_sync(kFull, v[j], bl);
            v[j] = fmaf(-l, pj, v[j]);
        }
        float pr = __shfl_sync(kFull, rhs, bl);
        rhs = fmaf(-l, pr, rhs);
        if (lane == bl) {
            active = false;
            ord = k;
            upiv = pv;
        }
    }
    // Back substitution in pivot order: the row eliminated at step k holds
    // the k-th row of the upper factor, whose diagonal is that lane's pivot;
    // every lane takes the reciprocal of its own pivot at once.
    const float uinv = 1.0f / upiv;
    float out = 0.f;
#pragma unroll
    for (int k = F - 1; k >= 0; --k) {
        unsigned owner = __ballot_sync(kFull, ord == k);
        int src = __ffs(owner) - 1;
        float mine = (ord == k) ? rhs * uinv : 0.f;
        float xk = __shfl_sync(kFull, mine, src);
        if (lane == k) out = xk;
        rhs = fmaf(-v[k], xk, rhs);
    }
    flags = 0;
    ratio = (f > 0) ? pmax / pmin : 1.f;
    if (singular) {
        flags = FLAG_SINGULAR | FLAG_RATIO;
        out = 0.f;
        ratio = __int_as_float(0x7f800000);
    } else if (!(ratio <= ratio_max)) {
        flags = FLAG_RATIO;
    }
    x_lane = out;
}

// ---------------------------------------------------------------------------
// Exact radix select of the s-th largest key, 8 bits per pass from the top of
// the magnitude key (bit 31 is always 0): pass 0 resolves the exponent
// (bits 30..23), passes 1-3 the mantissa (22..15, 14..7, 6..0). After a pass
// every key whose covered bits exceed the prefix P is kept; keys equal to P on
// the covered bits form the open class, of which `need` are still kept.
__device__ __forceinline__ int radix_shift(int pass) { return pass == 0 ? 23 : (pass == 1 ? 15 : (pass == 2 ? 7 : 0)); }
__device__ __forceinline__ uint32_t radix_before(int pass) {
    return pass == 0 ? 0u : (pass == 1 ? 0xff800000u : (pass == 2 ? 0xffff8000u : 0xffffff80u));
}
__device__ __forceinline__ uint32_t radix_after(int pass) {
    return pass == 0 ? 0xff800000u : (pass == 1 ? 0xffff8000u : (pass == 2 ? 0xffffff80u : 0xffffffffu));
}
__device__ __forceinline__ uint32_t radix_digit(uint32_t key, int pass) { return (key >> radix_shift(pass)) & 0xffu; }

struct BinPick {
    int digit;         // bin holding the need-th largest key
    uint32_t newneed;  // keys still to take inside that bin
    uint32_t inbin;    // keys in that bin
};

// Shared-memory histogram layout: bin b of column a at a * kHistRow + b +
// b / 32. Lanes working on different columns with the same bin hit banks
// 9a + ... (distinct, 9 is odd), and a lane reading its 8 consecutive bins
// 8l..8l+7 hits bank 8l + l/4 + q (distinct over the 32 lanes).
constexpr int kHistRow = 265;
__device__ __forceinline__ int hist_slot(int b) { return b + (b >> 5); }

// Warp-cooperative scan of 256 contiguous, 16-byte aligned global bins from
// the top bin down: the bin where the running count first reaches `need`
// (>= 1; the bins must hold at least `need` keys in total). The bins are
// cleared after reading.
__device__ __forceinline__ BinPick warp_pick_bin(uint32_t* bins, uint32_t need) {
    const int lane = threadIdx.x & 31;
    // Lane l holds bins 8l..8l+7: two 16-byte loads through L2 (other CTAs'
    // atomics made the counts), then two 16-byte stores of zero.
    uint4* quad = reinterpret_cast<uint4*>(bins) + 2 * lane;
    const uint4 lo4 = __ldcg(quad), hi4 = __ldcg(quad + 1);
    quad[0] = make_uint4(0u, 0u, 0u, 0u);
    quad[1] = make_uint4(0u, 0u, 0u, 0u);
    const uint32_t c[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
    const uint32_t lsum = c[0] + c[1] + c[2] + c[3] + c[4] + c[5] + c[6] + c[7];
    uint32_t incl = lsum;  // keys in bins of lanes >= this lane
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_down_sync(kFull, incl, o);
        if (lane + o < 32) incl += t;
    }
    const uint32_t above = incl - lsum;
    const unsigned ob = __ballot_sync(kFull, above < need && need <= incl);
    const int L = __ffs(ob) - 1;
    BinPick r{0, 0u, 0u};
    if (lane == L) {
        uint32_t cum = above;
        bool found = false;
#pragma unroll
        for (int q = 7; q >= 0; --q) {
            if (!found && cum + c[q] >= need) {
                r.digit = lane * 8 + q;
                r.newneed = need - cum;
                r.inbin = c[q];
                found = true;
            }
            if (!found) cum += c[q];
        }
    }
    r.digit = __shfl_sync(kFull, r.digit, L < 0 ? 0 : L);
    r.newneed = __shfl_sync(kFull, r.newneed, L < 0 ? 0 : L);
    r.inbin = __shfl_sync(kFull, r.inbin, L < 0 ? 0 : L);
    return r;
}

// Keep rule of one column after selection: (key & Mk) > P, or equal to P on
// the covered bits and at a position below cut.
__device__ __forceinline__ bool keep_rule(uint32_t key, uint32_t P, uint32_t Mk, int pos, int cut) {
    const uint32_t kc = key & Mk;
    return kc > P || (kc == P && pos < cut);
}

__device__ __forceinline__ void fallback_push(const Fallback& fb, int flags, int64_t row) {
    if (fb.rows != nullptr && flags != 0) fb.rows[atomicAdd(fb.count, 1u)] = (int32_t)row;
}

__device__ __forceinline__ void record_flags(Counters* c, int flags, float ratio) {
    if (flags & FLAG_RATIO) atomicAdd(&c->flagged, 1ull);
    if (flags & FLAG_SINGULAR) atomicAdd(&c->singular, 1ull);
    else if (ratio > 0.f && ratio < __int_as_float(0x7f800000))
        atomicMax(&c->max_ratio_bits, __float_as_uint(ratio));
}

}  // namespace als
