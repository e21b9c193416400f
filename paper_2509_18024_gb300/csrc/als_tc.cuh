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
    static constexpr int KT = PREC == TC_TF32X3 ? 32 : 64;  // positions per staged chunk
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

// Bounded wait for the MMAs committed to `bar` (phase parity `phase`).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    uint32_t done = 0;
    for (long it = 0; it < (1l << 24) && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(phase)
            : "memory");
    }
    return done != 0;
}

// Allocate TMEM and init the barrier (all threads of the CTA; ends in a barrier).
template <int F, int PREC>
__device__ __forceinline__ void tc_setup(uint8_t* tiles, uint64_t* bar, uint32_t* tmem_slot, TcCtx& ctx) {
    using C = TcCfg<F, PREC>;
    const int tid = threadIdx.x, warp = tid >> 5;
    // Padding rows of A (>= F) and of B (> F) are zero for the whole kernel.
    uint32_t* t32 = reinterpret_cast<uint32_t*>(tiles);
    for (int e = tid; e < C::TILE_BYTES / 4; e += blockDim.x) t32[e] = 0u;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    ctx.tmem = *tmem_slot;
    ctx.phase = 0;
    ctx.ok = true;
}

template <int F, int PREC>
__device__ __forceinline__ void tc_teardown(const TcCtx& ctx) {
    using C = TcCfg<F, PREC>;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(ctx.tmem), "r"(C::TMEM_COLS));
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

// Accumulate positions [k_begin, k_end) of a staged tile into the TMEM
// accumulator (first == true starts it from zero). x: [*][F] row-major,
// mask: W words per position, r: ratings. All threads call it.
template <int F, int PREC, int W>
__device__ __forceinline__ void tc_accumulate(TcCtx& ctx, uint8_t* tiles, uint64_t* bar, const float (*x)[F],
                                              const uint32_t (*mask)[W], const float* r, int k_begin, int k_end,
                                              bool sym, bool first) {
    using C = TcCfg<F, PREC>;
    const int tid = threadIdx.x;
    uint8_t* A0 = tiles;
    uint8_t* B0 = tiles + C::A_BYTES;
    uint8_t* A1 = tiles + C::A_BYTES + C::B_BYTES;  // lo copies (split-TF32 only)
    uint8_t* B1 = A1 + C::A_BYTES;
    constexpr int KC = C::KC;
    constexpr int GROUPS = C::KT / KC;  // 16-byte rows per feature per chunk
    bool started = !first;
    for (int c0 = k_begin; c0 < k_end; c0 += C::KT) {
        // Operand rows: (feature or rhs row m, 16-byte group g). Rows 0..F-1
        // of A are masked features, rows 0..F-1 of B plain features (masked
        // for the symmetric variant), row F of B the ratings.
        for (int e = tid; e < (F + 1) * GROUPS; e += blockDim.x) {
            const int m = e % (F + 1), g = e / (F + 1);
            float va[8], vb[8], la[8], lb[8];
#pragma unroll
            for (int q = 0; q < KC; ++q) {
                const int k = c0 + g * KC + q;
                float xv = 0.f, keep = 0.f;
                if (k < k_end) {
                    if (m < F) {
                        xv = x[k][m];
                        keep = ((mask[k][m >> 5] >> (m & 31)) & 1u) ? 1.f : 0.f;
                    } else {
                        xv = r[k];
                        keep = 1.f;
                    }
                }
                const float a = keep * xv;
                const float b = (m < F && sym) ? a : xv;
                if (PREC == TC_TF32X3) {
                    const float ah = __uint_as_float(tf32_rna(a)), bh = __uint_as_float(tf32_rna(b));
                    va[q] = ah;
                    vb[q] = bh;
                    la[q] = __uint_as_float(tf32_rna(a - ah));
                    lb[q] = __uint_as_float(tf32_rna(b - bh));
                } else if (PREC == TC_TF32) {
                    va[q] = __uint_as_float(tf32_rna(a));
                    vb[q] = __uint_as_float(tf32_rna(b));
                } else {
                    va[q] = a;
                    vb[q] = b;
                }
            }
            if (m < F) put16<PREC>(A0 + C::off(C::M, m, g * KC), va, KC);
            put16<PREC>(B0 + C::off(C::N, m, g * KC), vb, KC);
            if (PREC == TC_TF32X3) {
                if (m < F) put16<PREC>(A1 + C::off(C::M, m, g * KC), la, KC);
                put16<PREC>(B1 + C::off(C::N, m, g * KC), lb, KC);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int ks = 0; ks < C::KT / C::KSTEP; ++ks) {
                // Two 16-byte K groups per instruction.
                const uint32_t koff_a = (uint32_t)(2 * ks) * (C::M / 8) * 128;
                const uint32_t koff_b = (uint32_t)(2 * ks) * (C::N / 8) * 128;
                const int nterm = PREC == TC_TF32X3 ? 3 : 1;
#pragma unroll
                for (int t = 0; t < nterm; ++t) {
                    // split-TF32 terms: hi*hi, hi*lo, lo*hi
                    const uint8_t* Ap = (t == 2) ? A1 : A0;
                    const uint8_t* Bp = (t == 1) ? B1 : B0;
                    const uint64_t ad = umma_desc(smem_addr(Ap) + koff_a, (C::M / 8) * 128, 128);
                    const uint64_t bd = umma_desc(smem_addr(Bp) + koff_b, (C::N / 8) * 128, 128);
                    const uint32_t acc = started ? 1u : 0u;
                    if (PREC == TC_BF16)
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(ctx.tmem),
                            "l"(ad), "l"(bd), "r"(C::IDESC), "r"(acc));
                    else
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(ctx.tmem),
                            "l"(ad), "l"(bd), "r"(C::IDESC), "r"(acc));
                    started = true;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(bar)));
        }
        started = true;
        // The tile is rewritten by the next chunk: wait until the MMAs read it.
        if (!mbar_wait(bar, ctx.phase)) ctx.ok = false;
        ctx.phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (!started && tid == 0) {
        // Nothing was accumulated (empty range): the caller reads zeros via
        // tc_store's `empty` flag.
    }
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

}  // namespace als
