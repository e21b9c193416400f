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
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "core_als.h"

namespace {

constexpr int kTile = 64;     // output tile
constexpr int kTileK = 16;    // reduction slice
constexpr int kThreads = 256; // 16 x 16 threads, 4 x 4 outputs each
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
template <bool TA, bool TB, typename TBv>
__global__ void __launch_bounds__(kThreads) k_gemm(int M, int N, int k0, int k1, const float* __restrict__ A, int lda,
                                                   const TBv* __restrict__ B, int ldb, const float* __restrict__ bias,
                                                   float* __restrict__ C, int ldc) {
    __shared__ float As[kTileK][kTile + 4];
    __shared__ float Bs[kTileK][kTile + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
    float acc[4][4] = {};
    for (int kb = k0; kb < k1; kb += kTileK) {
        for (int e = threadIdx.x; e < kTileK * kTile; e += kThreads) {
            const int kk = e / kTile, mm = e % kTile;
            const int k = kb + kk, m = m0 + mm;
            float v = 0.f;
            if (k < k1 && m < M) v = TA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
            As[kk][mm] = v;
            const int n = n0 + mm;
            float w = 0.f;
            if (k < k1 && n < N) w = (float)(TB ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n]);
            Bs[kk][mm] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTileK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty * 4 + q];
                b[q] = Bs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int t = 0; t < 4; ++t) acc[q][t] = fmaf(a[q], b[t], acc[q][t]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int m = m0 + ty * 4 + q;
        if (m >= M) continue;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int n = n0 + tx * 4 + t;
            if (n < N) C[(int64_t)m * ldc + n] = acc[q][t] + (bias ? bias[n] : 0.f);
        }
    }
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

dim3 gemm_grid(int M, int N) { return dim3((N + kTile - 1) / kTile, (M + kTile - 1) / kTile); }
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
    int64_t part_cap = 0;

    int64_t oW1() const { return 0; }
    int64_t ob1() const { return (int64_t)hid * in; }
    int64_t oW2() const { return ob1() + hid; }
    int64_t ob2() const { return oW2() + (int64_t)hid * hid; }
    int64_t oW3() const { return ob2() + hid; }
    int64_t ob3() const { return oW3() + (int64_t)out * hid; }
};

namespace {

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
    k_gemm<false, true, __nv_bfloat16><<<gemm_grid((int)rows, H), kThreads, 0, st>>>(
        (int)rows, H, 0, I, X, I, W + n->oW1(), I, n->w + n->ob1(), n->z1, H);
    k_gelu_inplace<<<blocks_for(rows * H), 256, 0, st>>>(n->h1, n->z1, rows * H);
    k_gemm<false, true, __nv_bfloat16><<<gemm_grid((int)rows, H), kThreads, 0, st>>>(
        (int)rows, H, 0, H, n->h1, H, W + n->oW2(), H, n->w + n->ob2(), n->z2, H);
    k_gelu_inplace<<<blocks_for(rows * H), 256, 0, st>>>(n->h2, n->z2, rows * H);
    k_gemm<false, true, __nv_bfloat16><<<gemm_grid((int)rows, O), kThreads, 0, st>>>(
        (int)rows, O, 0, H, n->h2, H, W + n->oW3(), H, n->w + n->ob3(), n->y, O);
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
        k_gemm<true, false, float><<<gemm_grid(NZ, KA), kThreads, 0, st>>>(
            NZ, KA, r0, r1, dZ, NZ, A, KA, nullptr, n->part + (int64_t)s * NZ * KA, KA);
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
    k_gemm<false, false, __nv_bfloat16><<<gemm_grid((int)rows, H), kThreads, 0, st>>>(
        (int)rows, H, 0, O, n->dy, O, W + n->oW3(), H, nullptr, n->d2, H);
    k_gelu_back<<<blocks_for(rows * H), 256, 0, st>>>(n->d2, n->d2, n->z2, rows * H);
    rc = weight_grad(n, rows, n->d2, H, n->h1, H, n->oW2(), n->ob2());
    if (rc) return rc;
    k_gemm<false, false, __nv_bfloat16><<<gemm_grid((int)rows, H), kThreads, 0, st>>>(
        (int)rows, H, 0, H, n->d2, H, W + n->oW2(), H, nullptr, n->d1, H);
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
              cudaMalloc(&n->wb, n->n_params * 2) == cudaSuccess && cudaMalloc(&n->loss, 8) == cudaSuccess;
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
    for (void* p : {(void*)n->w, (void*)n->m, (void*)n->v, (void*)n->g, (void*)n->wb, (void*)n->loss})
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
    return cudaStreamSynchronize(n->stream) == cudaSuccess ? ALS_OK : ALS_ERR_CUDA;
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
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) return ALS_ERR_CUDA;
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
        if (cudaMemcpyAsync(&l, n->loss, 8, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
            cudaStreamSynchronize(n->stream) != cudaSuccess)
            return ALS_ERR_CUDA;
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
