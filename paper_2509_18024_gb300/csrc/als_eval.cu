// Evaluation kernels: the objective of Eq. (object function) (Sec. 2.1), the
// relative errors ReMSE / P-ReMSE and the recommendation metrics Hit@k and
// NDCG@k of Sec. 5.1. Predicted ratings are FP32 dot products u_i . m_j
// accumulated by fmaf in feature order; every sum that leaves a thread is
// FP64 and reduced in a fixed order (fixed grids), so results repeat bit for
// bit from run to run.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "als_eval.h"

namespace als_eval {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// FP32 prediction u . m in feature order (the order the oracle ranks by).
__device__ __forceinline__ float predict(const float* __restrict__ u, const float* __restrict__ m, int f) {
    float acc = 0.f;
    for (int a = 0; a < f; ++a) acc = fmaf(u[a], m[a], acc);
    return acc;
}

// The same chain read as float4 when both rows are 16-byte aligned whole
// float4s (f % 4 == 0): identical products and order, fewer loads.
__device__ __forceinline__ float predict_vec(const float* __restrict__ u, const float* __restrict__ m, int f) {
    if ((f & 3) != 0 || ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(m)) & 15u) != 0)
        return predict(u, m, f);
    const float4* u4 = reinterpret_cast<const float4*>(u);
    const float4* m4 = reinterpret_cast<const float4*>(m);
    float acc = 0.f;
    for (int q = 0; q < f / 4; ++q) {
        const float4 x = __ldg(u4 + q), y = __ldg(m4 + q);
        acc = fmaf(x.x, y.x, acc);
        acc = fmaf(x.y, y.y, acc);
        acc = fmaf(x.z, y.z, acc);
        acc = fmaf(x.w, y.w, acc);
    }
    return acc;
}

// Block sum of one double per thread (256 threads), fixed tree order.
__device__ __forceinline__ double block_sum256(double v, double* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// Data term of the objective: sum over the training entries of one side's
// rows of (r_e - u_i . m_{j_e})^2. Entry-parallel, so that long rows do not
// serialise: warp w takes the contiguous entries [w C, (w + 1) C) (C a
// multiple of 32), lane l its entries w C + l + 32 t; each lane finds the row
// of its first entry by binary search of indptr and then walks forward.
__global__ void __launch_bounds__(256) k_obj_data(const int64_t* __restrict__ indptr,
                                                  const int32_t* __restrict__ indices,
                                                  const float* __restrict__ values, int64_t n_rows, int64_t n_cols,
                                                  int64_t nnz, const float* __restrict__ U,
                                                  const float* __restrict__ M, int f, double* __restrict__ partials) {
    __shared__ double red[256];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * 8;
    const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int64_t chunk = ((nnz + warps - 1) / warps + 31) / 32 * 32;
    const int64_t e0 = w * chunk + lane, e1 = min(nnz, (w + 1) * chunk);
    double acc = 0.0;
    if (e0 < e1 && n_rows > 0) {
        int64_t lo = 0, hi = n_rows;  // the row i with indptr[i] <= e0 < indptr[i + 1]
        for (int it = 0; it < 64 && hi - lo > 1; ++it) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (indptr[mid] <= e0) lo = mid;
            else hi = mid;
        }
        int64_t i = lo;
        for (int64_t e = e0; e < e1; e += 32) {
            while (i + 1 < n_rows && indptr[i + 1] <= e) ++i;
            const int32_t j = indices[e];
            if ((uint32_t)j >= (uint64_t)n_cols) continue;  // never read outside M
            const double d = (double)values[e] - (double)predict_vec(U + i * f, M + (int64_t)j * f, f);
            acc += d * d;
        }
    }
    const double s = block_sum256(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Penalty of one side: sum_i w_i |x_i|^2 with w_i = n_i (weighted lambda) or
// 1 (plain), summed element by element in FP64.
__global__ void __launch_bounds__(256) k_obj_reg(const int64_t* __restrict__ indptr, int64_t n_rows,
                                                 const float* __restrict__ X, int f, int plain,
                                                 double* __restrict__ partials) {
    __shared__ double red[256];
    double acc = 0.0;
    // Element-parallel (coalesced): element e of X belongs to row e / f.
    const int64_t total = n_rows * f;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (int64_t)gridDim.x * 256) {
        const int64_t i = e / f;
        const double x = (double)X[e];
        acc += (plain ? 1.0 : (double)(indptr[i + 1] - indptr[i])) * (x * x);
    }
    const double s = block_sum256(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// One warp sums `n` partials of each of `groups` consecutive groups (lane l
// takes l, l + 32, ... in order, then a fixed butterfly); out = sum_g coef_g
// * total_g with coef = {1, c1, c1, ...} when combine, else out[g] = total_g.
__global__ void k_sum_groups(const double* __restrict__ partials, int n, int groups, int combine, double c1,
                             double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    double comb = 0.0;
    for (int g = 0; g < groups; ++g) {
        double s = 0.0;
        for (int q = lane; q < n; q += 32) s += partials[(int64_t)g * n + q];
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (combine) comb += (g == 0 ? 1.0 : c1) * s;
        else if (lane == 0) out[g] = s;
    }
    if (combine && lane == 0) out[0] = comb;
}

// sum_E (r - u.m)^2 and sum_E r^2 over listed entries.
__global__ void __launch_bounds__(256) k_sse_norm(int64_t n, const int32_t* __restrict__ iu,
                                                  const int32_t* __restrict__ im, const float* __restrict__ r,
                                                  const float* __restrict__ U, const float* __restrict__ M, int f,
                                                  double* __restrict__ partials) {
    __shared__ double red[256];
    double se = 0.0, sr = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256) {
        const double d = (double)r[e] - (double)predict_vec(U + (int64_t)iu[e] * f, M + (int64_t)im[e] * f, f);
        se += d * d;
        sr += (double)r[e] * (double)r[e];
    }
    const double a = block_sum256(se, red);
    const double b = block_sum256(sr, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = a;
        partials[gridDim.x + blockIdx.x] = b;
    }
}

// (score, item) order of the lists: larger score first, lower item on ties.
__device__ __forceinline__ bool ahead(float s1, int j1, float s2, int j2) { return s1 > s2 || (s1 == s2 && j1 < j2); }

// Recommendation lists and their metrics. One CTA per user (grid-stride):
//   1. a bitmap of the user's training items in shared memory;
//   2. every thread scores items j = tid, tid + 256, ... that are not rated,
//      keeping its best kRankMaxK in registers (sorted, insertion);
//   3. K rounds of a CTA-wide argmax over the threads' list heads give the
//      user's top K in order;
//   4. thread 0 checks them against the user's relevant items (sorted CSR row,
//      binary search) and accumulates hit and DCG / IDCG in FP64.
// Per-CTA sums go to partials[b], partials[grid + b], partials[2 grid + b].
__global__ void __launch_bounds__(kRankThreads) k_rank(int64_t n_u, int64_t n_m, int f, const float* __restrict__ U,
                                                       const float* __restrict__ M,
                                                       const int64_t* __restrict__ tr_ip,
                                                       const int32_t* __restrict__ tr_ix,
                                                       const int64_t* __restrict__ rel_ip,
                                                       const int32_t* __restrict__ rel_ix, int K, int k_hit,
                                                       int k_ndcg, int32_t* __restrict__ topk_out,
                                                       double* __restrict__ partials) {
    constexpr int L = kRankMaxK;
    extern __shared__ __align__(16) uint32_t smem_u32[];
    const int W = (int)((n_m + 31) / 32);
    uint32_t* bits = smem_u32;
    float* su = reinterpret_cast<float*>(bits + W);
    float* ls = su + ((f + 3) & ~3);
    int* li = reinterpret_cast<int*>(ls + kRankThreads * L);
    __shared__ float w_s[kRankThreads / 32];
    __shared__ int w_j[kRankThreads / 32], w_t[kRankThreads / 32];
    __shared__ int s_top[L];
    __shared__ int s_win;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    double acc_hit = 0.0, acc_ndcg = 0.0, acc_n = 0.0;
    for (int64_t i = blockIdx.x; i < n_u; i += gridDim.x) {
        __syncthreads();
        for (int w = tid; w < W; w += kRankThreads) bits[w] = 0u;
        for (int a = tid; a < f; a += kRankThreads) su[a] = U[i * f + a];
        __syncthreads();
        for (int64_t e = tr_ip[i] + tid; e < tr_ip[i + 1]; e += kRankThreads) {
            const int32_t j = tr_ix[e];
            if ((uint32_t)j < (uint64_t)n_m) atomicOr(&bits[j >> 5], 1u << (j & 31));
        }
        __syncthreads();
        float ts[L];
        int ti[L];
#pragma unroll
        for (int q = 0; q < L; ++q) {
            ts[q] = -INFINITY;
            ti[q] = 0x7fffffff;
        }
        for (int64_t jj = tid; jj < n_m; jj += kRankThreads) {
            const int j = (int)jj;
            if ((bits[j >> 5] >> (j & 31)) & 1u) continue;
            const float sc = predict(su, M + jj * f, f);
            if (!ahead(sc, j, ts[L - 1], ti[L - 1])) continue;
            // Insert, keeping ts/ti sorted (register indices stay static).
            bool placed = false;
#pragma unroll
            for (int q = L - 1; q >= 0; --q) {
                if (!placed) {
                    if (q > 0 && ahead(sc, j, ts[q - 1], ti[q - 1])) {
                        ts[q] = ts[q - 1];
                        ti[q] = ti[q - 1];
                    } else {
                        ts[q] = sc;
                        ti[q] = j;
                        placed = true;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < L; ++q) {
            ls[tid * L + q] = ts[q];
            li[tid * L + q] = ti[q];
        }
        __syncthreads();
        int head = 0;
        for (int q = 0; q < K; ++q) {
            float cs = head < L ? ls[tid * L + head] : -INFINITY;
            int cj = head < L ? li[tid * L + head] : 0x7fffffff;
            int ct = tid;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const float os = __shfl_xor_sync(kFull, cs, o);
                const int oj = __shfl_xor_sync(kFull, cj, o);
                const int ot = __shfl_xor_sync(kFull, ct, o);
                if (ahead(os, oj, cs, cj) || (os == cs && oj == cj && ot < ct)) {
                    cs = os;
                    cj = oj;
                    ct = ot;
                }
            }
            if (lane == 0) {
                w_s[warp] = cs;
                w_j[warp] = cj;
                w_t[warp] = ct;
            }
            __syncthreads();
            if (tid == 0) {
                float bs = w_s[0];
                int bj = w_j[0], bt = w_t[0];
                for (int v = 1; v < kRankThreads / 32; ++v)
                    if (ahead(w_s[v], w_j[v], bs, bj)) {
                        bs = w_s[v];
                        bj = w_j[v];
                        bt = w_t[v];
                    }
                s_top[q] = bj == 0x7fffffff ? -1 : bj;
                s_win = bj == 0x7fffffff ? -1 : bt;
            }
            __syncthreads();
            if (tid == s_win) ++head;
        }
        if (topk_out != nullptr && tid < K) topk_out[i * K + tid] = s_top[tid];
        if (tid == 0) {
            const int64_t lo = rel_ip[i], hi = rel_ip[i + 1];
            if (hi > lo) {
                double h = 0.0, dcg = 0.0, idcg = 0.0;
                for (int p = 0; p < K; ++p) {
                    const int j = s_top[p];
                    bool is_rel = false;
                    if (j >= 0) {
                        int64_t a = lo, b = hi;  // first entry >= j
                        while (a < b) {
                            const int64_t mid = a + (b - a) / 2;
                            if (rel_ix[mid] < j) a = mid + 1;
                            else b = mid;
                        }
                        is_rel = a < hi && rel_ix[a] == j;
                    }
                    if (p < k_hit && is_rel) h = 1.0;
                    if (p < k_ndcg && is_rel) dcg += 1.0 / log2((double)p + 2.0);
                }
                for (int p = 0; p < k_ndcg && p < hi - lo; ++p) idcg += 1.0 / log2((double)p + 2.0);
                acc_hit += h;
                acc_ndcg += dcg / idcg;
                acc_n += 1.0;
            }
        }
    }
    if (tid == 0) {
        partials[blockIdx.x] = acc_hit;
        partials[gridDim.x + blockIdx.x] = acc_ndcg;
        partials[2 * gridDim.x + blockIdx.x] = acc_n;
    }
}

}  // namespace

cudaError_t objective(cudaStream_t st, const int64_t* u_indptr, const int32_t* u_indices, const float* u_values,
                      int64_t n_u, int64_t u_nnz, const int64_t* m_indptr, int64_t n_m, const float* U,
                      const float* M, int f, double lambda, int plain_reg, double* partials, double* out_dev) {
    k_obj_data<<<kBlocks, 256, 0, st>>>(u_indptr, u_indices, u_values, n_u, n_m, u_nnz, U, M, f, partials);
    k_obj_reg<<<kBlocks, 256, 0, st>>>(u_indptr, n_u, U, f, plain_reg, partials + kBlocks);
    k_obj_reg<<<kBlocks, 256, 0, st>>>(m_indptr, n_m, M, f, plain_reg, partials + 2 * kBlocks);
    k_sum_groups<<<1, 32, 0, st>>>(partials, kBlocks, 3, 1, lambda, out_dev);
    return cudaGetLastError();
}

cudaError_t sse_and_norm(cudaStream_t st, int64_t n, const int32_t* iu, const int32_t* im, const float* r,
                         const float* U, const float* M, int f, double* partials, double* out_dev) {
    k_sse_norm<<<kBlocks, 256, 0, st>>>(n, iu, im, r, U, M, f, partials);
    k_sum_groups<<<1, 32, 0, st>>>(partials, kBlocks, 2, 0, 0.0, out_dev);
    return cudaGetLastError();
}

size_t rank_smem_bytes(int64_t n_m, int f) {
    return (size_t)((n_m + 31) / 32) * 4 + (size_t)((f + 3) & ~3) * 4 + (size_t)kRankThreads * kRankMaxK * 8;
}

cudaError_t rank(cudaStream_t st, int grid, int64_t n_u, int64_t n_m, int f, const float* U, const float* M,
                 const int64_t* train_indptr, const int32_t* train_indices, const int64_t* rel_indptr,
                 const int32_t* rel_indices, int K, int k_hit, int k_ndcg, int32_t* topk_out, double* partials,
                 double* out_dev) {
    const size_t smem = rank_smem_bytes(n_m, f);
    cudaError_t e = cudaFuncSetAttribute(k_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_rank<<<grid, kRankThreads, smem, st>>>(n_u, n_m, f, U, M, train_indptr, train_indices, rel_indptr, rel_indices,
                                             K, k_hit, k_ndcg, topk_out, partials);
    k_sum_groups<<<1, 32, 0, st>>>(partials, grid, 3, 0, 0.0, out_dev);
    return cudaGetLastError();
}

}  // namespace als_eval
