// Learned warm start: per-row features and a 3-layer MLP with hand-written
// forward, backward and Adam kernels.
//
//   features of row i: [sum_j r_ij y_j / sum_j r_ij (n_f values), log(1 + n_i),
//                       mean_j r_ij]   (y_j: the other side's factor rows)
//   net: z1 = W1 x + b1, h1 = GELU(z1); z2 = W2 h1 + b2, h2 = GELU(z2);
//        y = W3 h2 + b3;  GELU(z) = z Phi(z) (exact, with erf).
//   loss: mean over rows and outputs of (y - t)^2.
// Weights are kept in FP32 (the optimiser's master copy) and rounded to BF16
// for the forward and backward products; activations and all sums are FP32.
// Reductions over rows (weight gradients, loss) are split into fixed blocks
// and summed in a fixed order, so results are deterministic.
//
// Every product runs on the tensor cores (tcgen05.mma kind::tf32, FP32
// accumulator in tensor memory): a BF16 weight is exact in TF32, and an FP32
// operand x is split as x = hi + lo with hi its TF32 rounding, so that
// W x = W hi + W lo, and A B = hi hi + hi lo + lo hi for two FP32 operands,
// which keeps the products at FP32 accuracy.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <type_traits>

#include "core_als.h"
#include "als_tc.cuh"

namespace {

constexpr int kSplitRows = 4096;  // rows per partial of a weight gradient

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    const float cdf = 0.5f * (1.f + erff(z * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * __expf(-0.5f * z * z);
    return cdf + z * pdf;
}

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]), A(m, k) = TA ? A[k][m] : A[m][k]
// (leading dimension lda), B(k, n) = TB ? B[n][k] : B[k][n] (ldb). B may be
// BF16 (weights). k runs over [k0, k1). Output row-major with ldc.
//
// One CTA of 128 threads per tile of 128 rows x up to 256 columns: per
// chunk of 32 k the threads convert their rows of A and B into the
// canonical K-major, no-swizzle core-matrix layout of als_tc.cuh (TF32 hi
// and lo parts), thread 0 issues the MMAs into the tile's TMEM accumulator
// and commits them to an mbarrier, and the CTA waits for it (bounded, 1 s of
// GPU time) before the next chunk. Warps 0..3 then read rows 32w..32w+31
// from TMEM lanes with tcgen05.ld, add the bias and store. A wait that runs
// out sets bit 0 of *err; the tile then stores nothing.
constexpr int kTcRows = 128, kTcCols = 256, kTcKc = 32;
template <bool TA, bool TB, typename TBv>
__global__ void __launch_bounds__(128) k_tc_gemm(int M, int N, int k0, int k1, const float* __restrict__ A, int lda,
                                                 const TBv* __restrict__ B, int ldb, const float* __restrict__ bias,
                                                 float* __restrict__ C, int ldc, unsigned* err) {
    using namespace als;
    constexpr bool BSPLIT = !std::is_same<TBv, __nv_bfloat16>::value;  // FP32 B: hi and lo parts
    constexpr int A_BYTES = kTcRows * kTcKc * 4, B_BYTES = kTcCols * kTcKc * 4;
    extern __shared__ __align__(1024) uint8_t smem_t[];
    uint8_t* Ah = smem_t;
    uint8_t* Al = Ah + A_BYTES;
    uint8_t* Bh = Al + A_BYTES;
    uint8_t* Bl = Bh + B_BYTES;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTcRows, n0 = blockIdx.y * kTcCols;
    const int nt = min(kTcCols, (N - n0 + 15) / 16 * 16);  // MMA N: multiple of 16
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"((uint32_t)kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
    // Byte offset of element (row r, k) in an operand tile of R rows (TF32: 4 k per 16-byte core row).
    auto off = [](int R, int r, int k) { return (uint32_t)((k >> 2) * (R >> 3) * 128 + (r >> 3) * 128 + (r & 7) * 16 + (k & 3) * 4); };
    uint32_t phase = 0;
    bool ok = true, first = true;
    for (int kb = k0; kb < k1; kb += kTcKc) {
        // A: thread t converts row t of the tile, 32 k.
        {
            const int m = m0 + tid;
            for (int g = 0; g < kTcKc / 4; ++g) {
                float h4[4], l4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = kb + 4 * g + q;
                    float x = 0.f;
                    if (m < M && k < k1) x = TA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
                    const float hi = __uint_as_float(tf32_rna(x));
                    h4[q] = hi;
                    l4[q] = __uint_as_float(tf32_rna(x - hi));
                }
                *reinterpret_cast<float4*>(Ah + off(kTcRows, tid, 4 * g)) = make_float4(h4[0], h4[1], h4[2], h4[3]);
                *reinterpret_cast<float4*>(Al + off(kTcRows, tid, 4 * g)) = make_float4(l4[0], l4[1], l4[2], l4[3]);
            }
        }
        // B: rows n = tid, tid + 128 of the tile, element (n, k) = B(k, n).
        for (int r = tid; r < nt; r += 128) {
            const int n = n0 + r;
            for (int g = 0; g < kTcKc / 4; ++g) {
                float h4[4], l4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = kb + 4 * g + q;
                    float x = 0.f;
                    if (n < N && k < k1) x = (float)(TB ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n]);
                    const float hi = __uint_as_float(tf32_rna(x));
                    h4[q] = hi;
                    l4[q] = __uint_as_float(tf32_rna(x - hi));
                }
                *reinterpret_cast<float4*>(Bh + off(nt, r, 4 * g)) = make_float4(h4[0], h4[1], h4[2], h4[3]);
                if (BSPLIT)
                    *reinterpret_cast<float4*>(Bl + off(nt, r, 4 * g)) = make_float4(l4[0], l4[1], l4[2], l4[3]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int ks = 0; ks < kTcKc / 8; ++ks) {
                const uint32_t ka = (uint32_t)(2 * ks) * (kTcRows / 8) * 128, kbo = (uint32_t)(2 * ks) * (nt / 8) * 128;
#pragma unroll
                for (int t = 0; t < (BSPLIT ? 3 : 2); ++t) {
                    const uint8_t* Ap = t == 1 ? Al : Ah;
                    const uint8_t* Bp = t == 2 ? Bl : Bh;
                    const uint64_t ad = umma_desc(smem_addr(Ap) + ka, (kTcRows / 8) * 128, 128);
                    const uint64_t bd = umma_desc(smem_addr(Bp) + kbo, (uint32_t)(nt / 8) * 128, 128);
                    const uint32_t accum = (first && ks == 0 && t == 0) ? 0u : 1u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&bar)));
        }
        first = false;
        // The next chunk overwrites the operands: wait for these MMAs.
        const bool done = mbar_wait(&bar, phase);
        if (done) phase ^= 1u;
        ok = __syncthreads_and(done) != 0;
        if (!ok) break;
    }
    if (!ok) {
        if (tid == 0) report_timeout(err);
        mbar_wait(&bar, phase);  // one more bounded wait before the accumulator is freed
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && !first) {
        const int m = m0 + 32 * warp + lane;
        for (int c0 = 0; c0 < nt; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (m < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n < N) C[(int64_t)m * ldc + n] = __uint_as_float(v[j]) + (bias ? bias[n] : 0.f);
                }
            }
        }
    } else if (ok && first) {  // empty k range: C = bias
        const int m = m0 + tid;
        if (m < M)
            for (int n = n0; n < min(N, n0 + kTcCols); ++n) C[(int64_t)m * ldc + n] = bias ? bias[n] : 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTcCols));
}

template <bool TA, bool TB, typename TBv>
void tc_gemm(cudaStream_t st, int M, int N, int k0, int k1, const float* A, int lda, const TBv* B, int ldb,
             const float* bias, float* C, int ldc, unsigned* err) {
    if (M <= 0 || N <= 0) return;
    constexpr size_t smem = 2 * (size_t)kTcRows * kTcKc * 4 + 2 * (size_t)kTcCols * kTcKc * 4;
    cudaFuncSetAttribute(k_tc_gemm<TA, TB, TBv>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const dim3 grid((M + kTcRows - 1) / kTcRows, (N + kTcCols - 1) / kTcCols);
    k_tc_gemm<TA, TB, TBv><<<grid, 128, smem, st>>>(M, N, k0, k1, A, lda, B, ldb, bias, C, ldc, err);
}

__global__ void k_gelu_inplace(float* __restrict__ H, const float* __restrict__ Z, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        H[e] = gelu(Z[e]);
}

// dZ = dH * GELU'(Z)
__global__ void k_gelu_back(float* __restrict__ dZ, const float* __restrict__ dH, const float* __restrict__ Z,
                            int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dZ[e] = dH[e] * gelu_grad(Z[e]);
}

// dY = 2 (Y - T) / (n * out); per-block partial of sum (Y - T)^2 in FP64.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, int64_t n, double scale,
                      float* __restrict__ dY, double* __restrict__ partial) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float d = Y[e] - T[e];
        dY[e] = (float)(2.0 * scale) * d;
        acc += (double)d * d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out[c] = sum over split partials (fixed order) of P[s][c]; for bias
// gradients the partial is a column sum over a block of rows.
__global__ void k_colsum_partial(const float* __restrict__ D, int rows, int cols, int rows_per, float* __restrict__ P) {
    const int s = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
        float acc = 0.f;
        const int r1 = min(rows, (s + 1) * rows_per);
        for (int r = s * rows_per; r < r1; ++r) acc += D[(int64_t)r * cols + c];
        P[(int64_t)s * cols + c] = acc;
    }
}

__global__ void k_sum_splits(const float* __restrict__ P, int splits, int64_t n, float* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < splits; ++s) acc += P[(int64_t)s * n + e];
        out[e] = acc;
    }
}

__global__ void k_sum_doubles(const double* __restrict__ p, int n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < n; ++q) s += p[q];
        *out = s;
    }
}

// Adam on the FP32 master weights, then the BF16 copy.
__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, float* __restrict__ m,
                       float* __restrict__ v, const float* __restrict__ g, int64_t n, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + (1.f - b1) * gi;
        const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        const float step = lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        w[e] -= step;
        wb[e] = __float2bfloat16_rn(w[e]);
    }
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        wb[e] = __float2bfloat16_rn(w[e]);
}

// Features, one warp per row.
__global__ void k_features(const int64_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                           const float* __restrict__ values, int64_t n_rows, int64_t n_cols,
                           const float* __restrict__ Y, int f, float* __restrict__ out) {
    // One warp per row; lanes take the row's entries lane, lane + 32, ...
    // and keep partial sums of up to 32 feature columns at a time, which meet
    // by a fixed butterfly (the same order every run).
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n_rows) return;
    const int64_t lo = indptr[i], hi = indptr[i + 1];
    const int n = (int)(hi - lo);
    float rs = 0.f;
    for (int64_t e = lo + lane; e < hi; e += 32) rs += values[e];
#pragma unroll
    for (int o = 16; o; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
    float* dst = out + i * (f + 2);
    for (int a0 = 0; a0 < f; a0 += 32) {
        const int na = min(32, f - a0);
        float acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = 0.f;
        for (int64_t e = lo + lane; e < hi; e += 32) {
            const int32_t j = indices[e];
            if ((uint32_t)j >= (uint64_t)n_cols) continue;
            const float v = values[e];
            const float* y = Y + (int64_t)j * f + a0;
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (q < na) acc[q] = fmaf(v, y[q], acc[q]);
        }
        float mine = 0.f;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            float t = acc[q];
#pragma unroll
            for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == q) mine = t;
        }
        if (lane < na) dst[a0 + lane] = (n > 0 && rs != 0.f) ? mine / rs : 0.f;
    }
    if (lane == 0) {
        dst[f] = logf(1.f + (float)n);
        dst[f + 1] = n > 0 ? rs / (float)n : 0.f;
    }
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }



}  // namespace

struct als_mlp {
    int in = 0, hid = 0, out = 0;
    cudaStream_t stream = nullptr;
    int64_t n_params = 0;
    float* w = nullptr;            // master weights [W1 b1 W2 b2 W3 b3]
    __nv_bfloat16* wb = nullptr;   // BF16 copy (biases included, unused)
    float* m = nullptr;
    float* v = nullptr;
    float* g = nullptr;            // gradient, same layout
    int64_t step = 0;
    // activation workspace for `cap` rows
    int64_t cap = 0;
    float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr, *d1 = nullptr,
          *d2 = nullptr, *part = nullptr;
    double* dpart = nullptr;
    double* loss = nullptr;
    unsigned* err = nullptr;       // bit 0: a bounded tensor-core wait ran out
    int64_t part_cap = 0;

    int64_t oW1() const { return 0; }
    int64_t ob1() const { return (int64_t)hid * in; }
    int64_t oW2() const { return ob1() + hid; }
    int64_t ob2() const { return oW2() + (int64_t)hid * hid; }
    int64_t oW3() const { return ob2() + hid; }
    int64_t ob3() const { return oW3() + (int64_t)out * hid; }
};

namespace {

int mlp_check(als_mlp* n) {
    unsigned e = 0;
    if (cudaMemcpyAsync(&e, n->err, 4, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
        return ALS_ERR_CUDA;
    if (e == 0) return ALS_OK;
    cudaMemsetAsync(n->err, 0, 4, n->stream);
    return ALS_ERR_TIMEOUT;
}

void mlp_free_work(als_mlp* n) {
    for (float* p : {n->z1, n->h1, n->z2, n->h2, n->y, n->dy, n->d1, n->d2, n->part})
        if (p) cudaFree(p);
    if (n->dpart) cudaFree(n->dpart);
    n->z1 = n->h1 = n->z2 = n->h2 = n->y = n->dy = n->d1 = n->d2 = n->part = nullptr;
    n->dpart = nullptr;
    n->cap = 0;
}

int mlp_work(als_mlp* n, int64_t rows) {
    if (rows <= n->cap) return ALS_OK;
    mlp_free_work(n);
    const int64_t H = n->hid, O = n->out;
    bool ok = cudaMalloc(&n->z1, rows * H * 4) == cudaSuccess && cudaMalloc(&n->h1, rows * H * 4) == cudaSuccess &&
              cudaMalloc(&n->z2, rows * H * 4) == cudaSuccess && cudaMalloc(&n->h2, rows * H * 4) == cudaSuccess &&
              cudaMalloc(&n->y, rows * O * 4) == cudaSuccess && cudaMalloc(&n->dy, rows * O * 4) == cudaSuccess &&
              cudaMalloc(&n->d1, rows * H * 4) == cudaSuccess && cudaMalloc(&n->d2, rows * H * 4) == cudaSuccess;
    const int64_t splits = (rows + kSplitRows - 1) / kSplitRows;
    const int64_t pc = splits * std::max<int64_t>(n->hid * std::max(n->in, n->hid), n->out * n->hid);
    ok = ok && cudaMalloc(&n->part, pc * 4) == cudaSuccess && cudaMalloc(&n->dpart, 4096 * 8) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        mlp_free_work(n);
        return ALS_ERR_OOM;
    }
    n->cap = rows;
    return ALS_OK;
}

// Splitmix64 -> uniform in (-1, 1).
double mlp_uniform(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((double)(z >> 11) + 0.5) / 9007199254740992.0 * 2.0 - 1.0;
}

int forward(als_mlp* n, int64_t rows, const float* X) {
    const int I = n->in, H = n->hid, O = n->out;
    cudaStream_t st = n->stream;
    const __nv_bfloat16* W = n->wb;
    tc_gemm<false, true, __nv_bfloat16>(st, (int)rows, H, 0, I, X, I, W + n->oW1(), I, n->w + n->ob1(), n->z1, H,
                                        n->err);
    k_gelu_inplace<<<blocks_for(rows * H), 256, 0, st>>>(n->h1, n->z1, rows * H);
    tc_gemm<false, true, __nv_bfloat16>(st, (int)rows, H, 0, H, n->h1, H, W + n->oW2(), H, n->w + n->ob2(), n->z2, H,
                                        n->err);
    k_gelu_inplace<<<blocks_for(rows * H), 256, 0, st>>>(n->h2, n->z2, rows * H);
    tc_gemm<false, true, __nv_bfloat16>(st, (int)rows, O, 0, H, n->h2, H, W + n->oW3(), H, n->w + n->ob3(), n->y, O,
                                        n->err);
    return cudaGetLastError() == cudaSuccess ? ALS_OK : ALS_ERR_CUDA;
}

// dW = dZ^T A over rows (split into fixed row blocks, summed in order) and
// db = column sums of dZ; writes into the gradient buffer at offsets.
int weight_grad(als_mlp* n, int64_t rows, const float* dZ, int NZ, const float* A, int KA, int64_t oW, int64_t ob) {
    cudaStream_t st = n->stream;
    const int splits = (int)((rows + kSplitRows - 1) / kSplitRows);
    for (int s = 0; s < splits; ++s) {
        const int r0 = s * kSplitRows, r1 = (int)std::min<int64_t>(rows, (int64_t)(s + 1) * kSplitRows);
        // P[s] (NZ x KA) = dZ[r0:r1]^T A[r0:r1]
        tc_gemm<true, false, float>(st, NZ, KA, r0, r1, dZ, NZ, A, KA, nullptr, n->part + (int64_t)s * NZ * KA, KA,
                                    n->err);
    }
    k_sum_splits<<<blocks_for((int64_t)NZ * KA), 256, 0, st>>>(n->part, splits, (int64_t)NZ * KA, n->g + oW);
    // bias: column sums of dZ
    k_colsum_partial<<<dim3((NZ + 255) / 256, splits), 256, 0, st>>>(dZ, (int)rows, NZ, kSplitRows, n->part);
    k_sum_splits<<<blocks_for(NZ), 256, 0, st>>>(n->part, splits, NZ, n->g + ob);
    return cudaGetLastError() == cudaSuccess ? ALS_OK : ALS_ERR_CUDA;
}

int backward(als_mlp* n, int64_t rows, const float* X, const float* T) {
    const int I = n->in, H = n->hid, O = n->out;
    cudaStream_t st = n->stream;
    const __nv_bfloat16* W = n->wb;
    const int nb = 256;
    k_mse<<<nb, 256, 0, st>>>(n->y, T, rows * O, 1.0 / ((double)rows * O), n->dy, n->dpart);
    k_sum_doubles<<<1, 32, 0, st>>>(n->dpart, nb, n->loss);
    int rc = weight_grad(n, rows, n->dy, O, n->h2, H, n->oW3(), n->ob3());
    if (rc) return rc;
    // d h2 = dy W3 -> dz2
    tc_gemm<false, false, __nv_bfloat16>(st, (int)rows, H, 0, O, n->dy, O, W + n->oW3(), H, nullptr, n->d2, H, n->err);
    k_gelu_back<<<blocks_for(rows * H), 256, 0, st>>>(n->d2, n->d2, n->z2, rows * H);
    rc = weight_grad(n, rows, n->d2, H, n->h1, H, n->oW2(), n->ob2());
    if (rc) return rc;
    tc_gemm<false, false, __nv_bfloat16>(st, (int)rows, H, 0, H, n->d2, H, W + n->oW2(), H, nullptr, n->d1, H, n->err);
    k_gelu_back<<<blocks_for(rows * H), 256, 0, st>>>(n->d1, n->d1, n->z1, rows * H);
    return weight_grad(n, rows, n->d1, H, X, I, n->oW1(), n->ob1());
}

}  // namespace

extern "C" {

int als_mlp_create(als_mlp** out, int in_dim, int hidden, int out_dim, uint64_t seed, void* stream) {
    if (!out || in_dim < 1 || hidden < 1 || out_dim < 1) return ALS_ERR_ARG;
    *out = nullptr;
    als_mlp* n = new als_mlp();
    n->in = in_dim;
    n->hid = hidden;
    n->out = out_dim;
    n->stream = reinterpret_cast<cudaStream_t>(stream);
    n->n_params = n->ob3() + out_dim;
    const size_t b = n->n_params * 4;
    bool ok = cudaMalloc(&n->w, b) == cudaSuccess && cudaMalloc(&n->m, b) == cudaSuccess &&
              cudaMalloc(&n->v, b) == cudaSuccess && cudaMalloc(&n->g, b) == cudaSuccess &&
              cudaMalloc(&n->wb, n->n_params * 2) == cudaSuccess && cudaMalloc(&n->loss, 8) == cudaSuccess &&
              cudaMalloc(&n->err, 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        delete n;
        return ALS_ERR_OOM;
    }
    // Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases.
    std::vector<float> h(n->n_params, 0.f);
    auto fill = [&](int64_t off, int rows, int cols) {
        const double a = 1.0 / std::sqrt((double)cols);
        for (int64_t e = 0; e < (int64_t)rows * cols; ++e) h[off + e] = (float)(a * mlp_uniform(seed, off + e));
    };
    fill(n->oW1(), hidden, in_dim);
    fill(n->oW2(), hidden, hidden);
    fill(n->oW3(), out_dim, hidden);
    cudaMemcpy(n->w, h.data(), b, cudaMemcpyHostToDevice);
    cudaMemset(n->m, 0, b);
    cudaMemset(n->v, 0, b);
    cudaMemset(n->err, 0, 4);
    k_to_bf16<<<blocks_for(n->n_params), 256>>>(n->w, n->wb, n->n_params);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return ALS_ERR_CUDA;
    }
    *out = n;
    return ALS_OK;
}

int als_mlp_destroy(als_mlp* n) {
    if (!n) return ALS_ERR_ARG;
    cudaStreamSynchronize(n->stream);
    mlp_free_work(n);
    for (void* p : {(void*)n->w, (void*)n->m, (void*)n->v, (void*)n->g, (void*)n->wb, (void*)n->loss, (void*)n->err})
        if (p) cudaFree(p);
    delete n;
    return ALS_OK;
}

int64_t als_mlp_num_params(const als_mlp* n) { return n ? n->n_params : 0; }

int als_mlp_set_params(als_mlp* n, const float* params_host) {
    if (!n || !params_host) return ALS_ERR_ARG;
    if (cudaMemcpyAsync(n->w, params_host, n->n_params * 4, cudaMemcpyHostToDevice, n->stream) != cudaSuccess)
        return ALS_ERR_CUDA;
    k_to_bf16<<<blocks_for(n->n_params), 256, 0, n->stream>>>(n->w, n->wb, n->n_params);
    n->step = 0;
    cudaMemsetAsync(n->m, 0, n->n_params * 4, n->stream);
    cudaMemsetAsync(n->v, 0, n->n_params * 4, n->stream);
    return cudaStreamSynchronize(n->stream) == cudaSuccess ? ALS_OK : ALS_ERR_CUDA;
}

int als_mlp_get_params(als_mlp* n, float* params_host) {
    if (!n || !params_host) return ALS_ERR_ARG;
    if (cudaMemcpyAsync(params_host, n->w, n->n_params * 4, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess)
        return ALS_ERR_CUDA;
    return mlp_check(n);
}

int als_mlp_forward(als_mlp* n, int64_t rows, const float* X, float* Y) {
    if (!n || rows < 0 || (rows > 0 && (!X || !Y))) return ALS_ERR_ARG;
    if (rows == 0) return ALS_OK;
    int rc = mlp_work(n, rows);
    if (rc) return rc;
    rc = forward(n, rows, X);
    if (rc) return rc;
    return cudaMemcpyAsync(Y, n->y, rows * n->out * 4, cudaMemcpyDeviceToDevice, n->stream) == cudaSuccess
               ? ALS_OK
               : ALS_ERR_CUDA;
}

int als_mlp_grad(als_mlp* n, int64_t rows, const float* X, const float* T, float* grads_host, double* loss_host) {
    if (!n || rows <= 0 || !X || !T) return ALS_ERR_ARG;
    int rc = mlp_work(n, rows);
    if (!rc) rc = forward(n, rows, X);
    if (!rc) rc = backward(n, rows, X, T);
    if (rc) return rc;
    if (grads_host && cudaMemcpyAsync(grads_host, n->g, n->n_params * 4, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess)
        return ALS_ERR_CUDA;
    double l = 0.0;
    if (cudaMemcpyAsync(&l, n->loss, 8, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess) return ALS_ERR_CUDA;
    rc = mlp_check(n);
    if (rc) return rc;
    if (loss_host) *loss_host = l / ((double)rows * n->out);
    return ALS_OK;
}

int als_mlp_train_step(als_mlp* n, int64_t rows, const float* X, const float* T, float lr, double* loss_host) {
    if (!n || rows <= 0 || !X || !T || !(lr > 0.f)) return ALS_ERR_ARG;
    int rc = mlp_work(n, rows);
    if (!rc) rc = forward(n, rows, X);
    if (!rc) rc = backward(n, rows, X, T);
    if (rc) return rc;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - std::pow(b1, (float)n->step), bc2 = 1.f - std::pow(b2, (float)n->step);
    k_adam<<<blocks_for(n->n_params), 256, 0, n->stream>>>(n->w, n->wb, n->m, n->v, n->g, n->n_params, lr, b1, b2,
                                                           1e-8f, bc1, bc2);
    if (cudaGetLastError() != cudaSuccess) return ALS_ERR_CUDA;
    if (loss_host) {
        double l = 0.0;
        if (cudaMemcpyAsync(&l, n->loss, 8, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess) return ALS_ERR_CUDA;
        rc = mlp_check(n);
        if (rc) return rc;
        *loss_host = l / ((double)rows * n->out);
    }
    return ALS_OK;
}

int als_features(const als_csr* R, const float* Y, int n_f, float* feat, void* stream) {
    if (!R || n_f < 1 || (R->n_rows > 0 && (!Y || !feat))) return ALS_ERR_ARG;
    if (R->n_rows == 0) return ALS_OK;
    const int64_t threads = R->n_rows * 32;
    k_features<<<(int)((threads + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        R->indptr, R->indices, R->values, R->n_rows, R->n_cols, Y, n_f, feat);
    return cudaGetLastError() == cudaSuccess ? ALS_OK : ALS_ERR_CUDA;
}

}  // extern "C"
