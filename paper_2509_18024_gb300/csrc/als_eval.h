// Host launchers of the evaluation kernels (als_eval.cu): the objective of
// Eq. (object function), the relative errors of Sec. 5.1 (ReMSE / P-ReMSE)
// and the recommendation metrics Hit@k / NDCG@k. Every launcher enqueues on
// `st` and returns the launch status; the C ABI in als_api.cu owns the
// buffers and the handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace als_eval {

constexpr int kBlocks = 608;    // partial sums per reduction (fixed grid, fixed order)
constexpr int kRankMaxK = 16;   // longest recommendation list
constexpr int kRankThreads = 256;

// Partials needed by objective(): 3 * kBlocks doubles, plus 1 for the result.
// out_dev = data term + lambda * (penalty of U + penalty of M).
cudaError_t objective(cudaStream_t st, const int64_t* u_indptr, const int32_t* u_indices, const float* u_values,
                      int64_t n_u, int64_t u_nnz, const int64_t* m_indptr, int64_t n_m, const float* U,
                      const float* M, int f, double lambda, int plain_reg, double* partials, double* out_dev);

// Partials: 2 * kBlocks doubles. out_dev[0] = sum_E (r - u.m)^2, out_dev[1] = sum_E r^2.
cudaError_t sse_and_norm(cudaStream_t st, int64_t n, const int32_t* iu, const int32_t* im, const float* r,
                         const float* U, const float* M, int f, double* partials, double* out_dev);

// Shared memory of the ranking kernel for n_m items and rank f.
size_t rank_smem_bytes(int64_t n_m, int f);

// Recommendation lists (K <= kRankMaxK) and metrics. partials: 3 * grid
// doubles; out_dev[0..2] = (sum of hits, sum of NDCG, users evaluated).
cudaError_t rank(cudaStream_t st, int grid, int64_t n_u, int64_t n_m, int f, const float* U, const float* M,
                 const int64_t* train_indptr, const int32_t* train_indices, const int64_t* rel_indptr,
                 const int32_t* rel_indices, int K, int k_hit, int k_ndcg, int32_t* topk_out, double* partials,
                 double* out_dev);

}  // namespace als_eval
