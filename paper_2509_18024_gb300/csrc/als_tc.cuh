// Tensor-core (tcgen05) assembly of the masked normal equations of Eq. core_ui:
//   D[a][c] = sum_k A[a][k] B[c][k],  A = X*^T (features x positions, masked),
//   B = [X | r]^T (features + rhs column), so D[:, :F] = X*^T X and
//   D[:, F] = X*^T r.
// Operands live in shared memory in the canonical K-major layout without
// swizzle (core matrices of 8 rows x 16 bytes), one thread issues
// tcgen05.mma with M = 128 (rows >= F of A are zero) and N = F + 16, the
// accumulator stays in tensor memory, and warps 0..3 read it back with
// tcgen05.ld (row a of D in TMEM lane a).
//
// Precisions: BF16 (kind::f16), TF32 (kind::tf32), and an FP32-accurate
// split-TF32 mode where x = x_hi + x_lo (x_hi = TF32 rounding of x) and
// hi*hi + hi*lo + lo*hi are accumulated into the same FP32 accumulator.
#pragma once

#include <cuda_bf16.h>

#include "als_device.cuh"

namespace als {

enum { TC_BF16 = 0, TC_TF32 = 1, TC_TF32X3 = 2 };

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor (no swizzle): start address,
// leading (K-direction) and stride (8-row-group) byte offsets, version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3fff);
    d |= (uint64_t)((lbo >> 4) & 0x3fff) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3fff) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

template <int F, int PREC>
struct TcCfg {
    static constexpr int M = 128;
    static constexpr int N = F + 16;                 // G columns + rhs column, multiple of 16
    static constexpr int ESZ = PREC == TC_BF16 ? 2 : 4;
    static constexpr int KC = 16 / ESZ;              // elements per 16-byte core-matrix row
    static constexpr int KSTEP = 32 / ESZ;           // K of one instruction (32 bytes)
    // positions per staged chunk (two tile buffers must fit with the slice)
    static constexpr int KT = PREC == TC_BF16 ? 64 : (PREC == TC_TF32 ? 32 : 16);
    static constexpr int NSPLIT = PREC == TC_TF32X3 ? 2 : 1;  // hi (and lo) copies
    static constexpr int A_BYTES = M * KT * ESZ;
    static constexpr int B_BYTES = N * KT * ESZ;
    static constexpr int TILE_BYTES = NSPLIT * (A_BYTES + B_BYTES);
    static constexpr uint32_t TMEM_COLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
    static constexpr uint32_t IDESC = (1u << 4) | ((PREC == TC_BF16 ? 1u : 2u) << 7) |
                                      ((PREC == TC_BF16 ? 1u : 2u) << 10) | ((uint32_t)(N >> 3) << 17) |
                                      ((uint32_t)(M >> 4) << 24);
    // Byte offset of element (row m, position k) in an R-row operand tile.
    __device__ static __forceinline__ uint32_t off(int R, int m, int k) {
        return (uint32_t)((k / KC) * (R / 8) * 128 + (m / 8) * 128 + (m % 8) * 16 + (k % KC) * ESZ);
    }
};

// Per-CTA tensor-core state: TMEM accumulator and the completion barrier.
struct TcCtx {
    uint32_t tmem;   // TMEM base address of the accumulator
    uint32_t phase;  // parity of the next mbarrier phase to wait for
    bool ok;         // false once a bounded wait ran out
};

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase parity `phase` of `bar` (the MMAs committed to it):
// gives up after limit_ns of global time and returns false.
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s; an MMA batch completes in microseconds
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, uint64_t limit_ns = kWaitLimitNs) {
    uint32_t done = 0;
    const uint64_t t0 = global_ns();
    for (;;) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(phase)
            : "memory");
        if (done || global_ns() - t0 > limit_ns) break;
    }
    return done != 0;
}

// Records a bounded wait that ran out in the sticky device error word.
constexpr unsigned kDevErrTimeout = 1u;
__device__ __forceinline__ void report_timeout(unsigned* err) {
    if (err) atomicOr(err, kDevErrTimeout);
}

// Stages n floats from global src to shared dst, all threads calling. When
// both addresses are 16-byte aligned and 4 n is a multiple of 16, thread 0
// issues one bulk copy (cp.async.bulk, completing on `bar`, a one-arrival
// barrier whose next phase has parity `phase`) and waits for it with the 1 s
// bound; otherwise a strided loop copies. Returns false (CTA-uniform) if the
// wait ran out; that copy then gets one more bounded wait, and bit 0 of err
// is set.
__device__ __forceinline__ bool stage_block(float* dst, const float* src, int n, uint64_t* bar, uint32_t& phase,
                                            unsigned* err) {
    const bool bulk = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 &&
                      (n & 3) == 0;
    bool ok = true;
    if (!bulk) {
        for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
    } else if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)n * 4u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_addr(dst)),
                     "l"(src), "r"(bytes), "r"(smem_addr(bar))
                     : "memory");
        ok = mbar_wait(bar, phase);
        if (!ok) {
            report_timeout(err);
            (void)mbar_wait(bar, phase);
        }
        phase ^= 1u;
    }
    return __syncthreads_and(ok) != 0;
}

// Warp-level form of stage_block for a warp's own system: lane 0 sets up the
// warp's barrier, issues the bulk copy and waits for it (1 s bound); the
// strided copy when the addresses or size do not allow a bulk copy. Returns
// false (warp-uniform) if the wait ran out, after a second bounded wait.
__device__ __forceinline__ bool stage_warp(float* dst, const float* src, int n, uint64_t* bar, unsigned* err) {
    const int lane = threadIdx.x & 31;
    const bool bulk = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 &&
                      (n & 3) == 0;
    bool ok = true;
    if (!bulk) {
        for (int e = lane; e < n; e += 32) dst[e] = src[e];
    } else if (lane == 0) {
        const uint32_t bytes = (uint32_t)n * 4u;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_addr(dst)),
                     "l"(src), "r"(bytes), "r"(smem_addr(bar))
                     : "memory");
        ok = mbar_wait(bar, 0u);
        if (!ok) {
            report_timeout(err);
            (void)mbar_wait(bar, 0u);
        }
    }
    __syncwarp();
    return __all_sync(0xffffffffu, ok) != 0;
}

// Self-test of the bounded wait: thread 0 waits on a fresh barrier that
// nothing arrives at, so the wait runs out after limit_ns and is recorded in
// the error word exactly as a timeout of the tensor-core pipelines is.
static __global__ void k_wait_selftest(uint64_t limit_ns, unsigned* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
        if (!mbar_wait(&bar, 0u, limit_ns)) report_timeout(err);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&bar)));
    }
}

// Write one 16-byte operand row (KC consecutive positions of one feature).
template <int PREC>
__device__ __forceinline__ void put16(uint8_t* dst, const float (&v)[8], int kc) {
    if (PREC == TC_BF16) {
        __nv_bfloat162 p[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) p[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(p);
    } else {
        uint4 u;
        u.x = __float_as_uint(v[0]);
        u.y = __float_as_uint(v[1]);
        u.z = __float_as_uint(v[2]);
        u.w = __float_as_uint(v[3]);
        *reinterpret_cast<uint4*>(dst) = u;
    }
    (void)kc;
}

// Read the accumulator rows 0..F-1, columns 0..F (G and rhs) and hand each
// value to store(a, c, v). Warps 0..3 (lanes = TMEM rows) take part.
template <int F, int PREC, class Store>
__device__ __forceinline__ void tc_store(const TcCtx& ctx, bool empty, Store store) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= 4 || 32 * warp >= F) return;
    const int a = 32 * warp + lane;
#pragma unroll 1
    for (int c0 = 0; c0 <= F; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = ctx.tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (a < F) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (c0 + j <= F) store(a, c0 + j, (empty || !ctx.ok) ? 0.f : __uint_as_float(v[j]));
        }
    }
}

// Floats of the transpose buffer tc_store_rows needs (32 x 17 per warp, warps 0..3).
constexpr int kTcStoreBufFloats = 4 * 32 * 17;

// Same values as tc_store, handed to store(a, c, v) in an order where the
// lanes of a warp take 16 consecutive columns of two rows: each warp passes
// its 32 x 16 block through a 32 x 17 transpose buffer (tbuf, warp w at
// w * 32 * 17), so that stores into a row-major [F][F + 1] block coalesce.
template <int F, int PREC, class Store>
__device__ __forceinline__ void tc_store_rows(const TcCtx& ctx, bool empty, Store store, float* tbuf) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= 4 || 32 * warp >= F) return;
    float* T = tbuf + warp * 32 * 17;
#pragma unroll 1
    for (int c0 = 0; c0 <= F; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = ctx.tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int j = 0; j < 16; ++j) T[lane * 17 + j] = (empty || !ctx.ok) ? 0.f : __uint_as_float(v[j]);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int rr = 2 * i + (lane >> 4), jj = lane & 15;
            const int a = 32 * warp + rr, c = c0 + jj;
            if (a < F && c <= F) store(a, c, T[rr * 17 + jj]);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Pipelined, persistent form: two operand tile buffers (each with its own
// completion barrier) and one TMEM accumulator. Converting chunk c + 1 runs
// while the MMAs of chunk c execute; a buffer is rewritten only after the
// commit that last read it completed, so no barrier ever runs two phases
// ahead of its waiter. A row's (or run's) accumulator is read back before
// the next row's first MMA is issued, after that row has been staged and
// selected, so one accumulator keeps the overlap and leaves tensor memory
// for a second CTA per SM.
constexpr int kTcAccums = 1;
struct TcPipe {
    uint32_t tmem;    // base of the two accumulators
    uint32_t ph[2];   // parity of the next completion per buffer
    int pend[2];      // a commit on this buffer is outstanding
    int next;         // buffer the next chunk uses
    bool ok;          // false once a bounded wait ran out
    unsigned* err;    // sticky device error word for such a timeout (or null)
};

template <int F, int PREC>
__device__ __forceinline__ void tc_pipe_setup(uint8_t* tiles, uint64_t* bars, uint32_t* tmem_slot, TcPipe& P,
                                              unsigned* err) {
    using C = TcCfg<F, PREC>;
    const int tid = threadIdx.x, warp = tid >> 5;
    uint32_t* t32 = reinterpret_cast<uint32_t*>(tiles);
    for (int e = tid; e < 2 * C::TILE_BYTES / 4; e += blockDim.x) t32[e] = 0u;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(kTcAccums * C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    P.tmem = *tmem_slot;
    P.ph[0] = P.ph[1] = 0u;
    P.pend[0] = P.pend[1] = 0;
    P.next = 0;
    P.ok = true;
    P.err = err;
}

// Wait for the last commit on buffer b. A wait that runs out records the
// timeout in the error word (the host returns ALS_ERR_TIMEOUT) and clears
// this thread's ok; the commit stays marked pending so that the teardown can
// give it one more bounded wait before the tensor memory is freed. Callers
// make ok uniform across the CTA at their next barrier.
__device__ __forceinline__ void tc_pipe_drain(TcPipe& P, uint64_t* bars, int b) {
    if (P.pend[b] && P.ok) {
        if (mbar_wait(&bars[b], P.ph[b])) {
            P.ph[b] ^= 1u;
            P.pend[b] = 0;
        } else {
            report_timeout(P.err);
            P.ok = false;
        }
    }
}

// One 16-byte group of operand rows: feature m (or the rhs, RHS) at the
// KC positions of group g of the tile starting at c0. A takes the masked
// value, B the unmasked one (asymmetric Gram; masked in the symmetric
// modes; the rhs unmasked), split into TF32 hi and lo in the split mode.
template <int F, int PREC, int W, bool RHS>
__device__ __forceinline__ void tc_conv_item(uint8_t* A0, uint8_t* B0, uint8_t* A1, uint8_t* B1,
                                             const float (*x)[xpitch(F)], const uint32_t (*mask)[W], const float* r,
                                             int n, bool sym, int c0, int m, int g) {
    using C = TcCfg<F, PREC>;
    constexpr int KC = C::KC;
    float va[8], vb[8], la[8], lb[8];
#pragma unroll
    for (int q = 0; q < KC; ++q) {
        const int k = c0 + g * KC + q;
        float xv = 0.f, keep = 0.f;
        if (k < n) {
            if (!RHS) {
                xv = x[k][m];
                keep = ((mask[k][m >> 5] >> (m & 31)) & 1u) ? 1.f : 0.f;
            } else {
                xv = r[k];
                keep = 1.f;
            }
        }
        const float a = keep * xv;
        const float bv = (!RHS && sym) ? a : xv;
        if (PREC == TC_TF32X3) {
            const float ah = __uint_as_float(tf32_rna(a)), bh = __uint_as_float(tf32_rna(bv));
            va[q] = ah;
            vb[q] = bh;
            la[q] = __uint_as_float(tf32_rna(a - ah));
            lb[q] = __uint_as_float(tf32_rna(bv - bh));
        } else if (PREC == TC_TF32) {
            va[q] = __uint_as_float(tf32_rna(a));
            vb[q] = __uint_as_float(tf32_rna(bv));
        } else {
            va[q] = a;
            vb[q] = bv;
        }
    }
    if (!RHS) put16<PREC>(A0 + C::off(C::M, m, g * KC), va, KC);
    put16<PREC>(B0 + C::off(C::N, m, g * KC), vb, KC);
    if (PREC == TC_TF32X3) {
        if (!RHS) put16<PREC>(A1 + C::off(C::M, m, g * KC), la, KC);
        put16<PREC>(B1 + C::off(C::N, m, g * KC), lb, KC);
    }
}

// Accumulate positions [0, n) of a staged tile into accumulator `acc`
// (0 or 1), starting it from zero when `fresh` (else adding to what it
// holds). All threads call it; MMAs stay in flight. Once a wait has run out
// (ok false, made CTA-uniform at the barrier before the issue) nothing is
// converted or issued any more.
template <int F, int PREC, int W>
__device__ __forceinline__ void tc_pipe_row(TcPipe& P, uint8_t* tiles, uint64_t* bars, const float (*x)[xpitch(F)],
                                            const uint32_t (*mask)[W], const float* r, int n, bool sym, int acc,
                                            bool fresh = true) {
    using C = TcCfg<F, PREC>;
    const int tid = threadIdx.x;
    constexpr int KC = C::KC;
    constexpr int GROUPS = C::KT / KC;
    const uint32_t dacc = P.tmem + (uint32_t)(acc & (kTcAccums - 1)) * C::TMEM_COLS;
    for (int c0 = 0; c0 < n; c0 += C::KT) {
        const int b = P.next;
        P.next ^= 1;
        tc_pipe_drain(P, bars, b);
        uint8_t* A0 = tiles + b * C::TILE_BYTES;
        uint8_t* B0 = A0 + C::A_BYTES;
        uint8_t* A1 = B0 + C::B_BYTES;
        uint8_t* B1 = A1 + C::A_BYTES;
        static_assert((F & (F - 1)) == 0, "tensor-core widths are powers of two");
        // Feature rows (F a power of two: the index split is a mask and a
        // shift, and no warp straddles the rhs), then the rhs row of B.
        if (P.ok) {
            for (int e = tid; e < F * GROUPS; e += blockDim.x)
                tc_conv_item<F, PREC, W, false>(A0, B0, A1, B1, x, mask, r, n, sym, c0, e & (F - 1), e / F);
            for (int g = tid; g < GROUPS; g += blockDim.x)
                tc_conv_item<F, PREC, W, true>(A0, B0, A1, B1, x, mask, r, n, sym, c0, F, g);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        P.ok = __syncthreads_and(P.ok) != 0;
        if (!P.ok) continue;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int ks = 0; ks < C::KT / C::KSTEP; ++ks) {
                const uint32_t koff_a = (uint32_t)(2 * ks) * (C::M / 8) * 128;
                const uint32_t koff_b = (uint32_t)(2 * ks) * (C::N / 8) * 128;
                const int nterm = PREC == TC_TF32X3 ? 3 : 1;
#pragma unroll
                for (int t = 0; t < nterm; ++t) {
                    const uint8_t* Ap = (t == 2) ? A1 : A0;
                    const uint8_t* Bp = (t == 1) ? B1 : B0;
                    const uint64_t ad = umma_desc(smem_addr(Ap) + koff_a, (C::M / 8) * 128, 128);
                    const uint64_t bd = umma_desc(smem_addr(Bp) + koff_b, (C::N / 8) * 128, 128);
                    const uint32_t accum = (!fresh || c0 > 0 || ks > 0 || t > 0) ? 1u : 0u;
                    if (PREC == TC_BF16)
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dacc),
                            "l"(ad), "l"(bd), "r"(C::IDESC), "r"(accum));
                    else
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dacc),
                            "l"(ad), "l"(bd), "r"(C::IDESC), "r"(accum));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&bars[b])));
        }
        P.pend[b] = 1;
    }
}

// Wait for every outstanding MMA, then read accumulator `acc` (rows 0..F-1,
// columns 0..F) into store(a, c, v); `empty` rows store zeros. With tbuf
// (kTcStoreBufFloats of free shared memory) the values go out in the
// coalescing order of tc_store_rows.
template <int F, int PREC, class Store>
__device__ __forceinline__ void tc_pipe_finish(TcPipe& P, uint64_t* bars, int acc, bool empty, Store store,
                                               float* tbuf = nullptr) {
    using C = TcCfg<F, PREC>;
    tc_pipe_drain(P, bars, 0);
    tc_pipe_drain(P, bars, 1);
    P.ok = __syncthreads_and(P.ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    TcCtx ctx;
    ctx.tmem = P.tmem + (uint32_t)(acc & (kTcAccums - 1)) * C::TMEM_COLS;
    ctx.phase = 0;
    ctx.ok = P.ok;
    if (tbuf != nullptr)
        tc_store_rows<F, PREC>(ctx, empty, store, tbuf);
    else
        tc_store<F, PREC>(ctx, empty, store);
}

// Free the accumulators. After a wait that ran out, each commit still marked
// pending gets one more bounded wait first (the MMAs it covers write the
// tensor memory that is about to be freed).
template <int F, int PREC>
__device__ __forceinline__ void tc_pipe_teardown(TcPipe& P, uint64_t* bars) {
    using C = TcCfg<F, PREC>;
    if (!P.ok)
        for (int b = 0; b < 2; ++b)
            if (P.pend[b] && mbar_wait(&bars[b], P.ph[b])) {
                P.ph[b] ^= 1u;
                P.pend[b] = 0;
            }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(P.tmem),
                     "r"(kTcAccums * C::TMEM_COLS));
}

}  // namespace als
