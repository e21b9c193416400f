/*
 * core_als.h - C ABI of the GB300 (sm_103a) core-elements ALS library.
 *
 * The method (Xue, Li, Zhang, Meng, "Core-elements Subsampling for
 * Alternating Least Squares", arXiv 2509.18024):
 *
 *   A rating matrix R (n_u x n_m) with missing entries is factorised as
 *   R ~ U M^T with rank n_f (Sec. 2.1). Each sweep of Algorithm 2 updates
 *   every user row, then every item row. For a row i with observed index set
 *   I_i (|I_i| = n_i), the design slice X = Y[I_i] (n_i x n_f) is made of the
 *   other side's factor rows in ascending index order, and
 *
 *     CES (Algorithm 1):  in every column a of X keep the s_i = floor(n_i r)
 *                         entries of largest |x_ka| and zero the rest: X*.
 *     Eq. (core_ui/mj):   x_i = (X*^T X + lambda n_i E)^{-1} X*^T r_i.
 *
 *   With budget r = 1 (or gram_mode ALS_GRAM_FULL) this is the full ALS
 *   update of Eq. (U format) / (M format).
 *
 * Conventions for every call:
 *   - Pointers are DEVICE pointers unless the parameter name ends in _host.
 *   - Matrices are row-major, FP32 unless stated; factor rows have n_f
 *     contiguous floats (row stride n_f).
 *   - A side of the rating matrix is passed as compressed rows (als_csr):
 *     the user side is R in CSR, the item side is R^T in CSR (= R in CSC).
 *     Indices inside a row must be sorted ascending and unique; values finite.
 *   - All work is enqueued on the handle's CUDA stream. Calls return when the
 *     work is enqueued, except where a _host output is filled (those
 *     synchronise the stream) and the first call on a new rating structure
 *     (see als_prepare). Inside a half-sweep the handle forks independent
 *     row groups onto side streams of its own (created on first use,
 *     destroyed with the handle) and joins them back into the handle's
 *     stream before the call's work ends on it: ordering against other work
 *     on the handle's stream, and graph capture of that stream, are as if
 *     everything ran on it.
 *   - The caller owns every buffer passed in; the library never frees caller
 *     memory. The handle owns its workspace (als_workspace_bytes).
 *   - Return value: ALS_OK (0) or a negative ALS_ERR_* code. Nothing is
 *     written to outputs after an argument error. als_status_string() names
 *     a code; als_last_error() gives the handle's last message.
 */
#ifndef CORE_ALS_H
#define CORE_ALS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ALS_OK 0
#define ALS_ERR_ARG (-1)            /* bad argument (null pointer, size, option) */
#define ALS_ERR_CSR (-2)            /* unsorted, duplicate or out-of-range index, bad indptr */
#define ALS_ERR_NONFINITE (-3)      /* NaN/Inf rating value */
#define ALS_ERR_CUDA (-4)           /* a CUDA runtime call failed */
#define ALS_ERR_TIMEOUT (-5)        /* a bounded device wait ran out */
#define ALS_ERR_OOM (-6)            /* device allocation failed or workspace cap hit */
#define ALS_ERR_DEVICE_BOUNDS (-7)  /* a device-side bounds check fired */
#define ALS_ERR_UNSUPPORTED (-8)    /* option combination not built (e.g. n_f > 128) */

/* Regulariser: weighted lambda n_i (Eq. object function) or plain lambda. */
#define ALS_REG_WEIGHTED 0
#define ALS_REG_PLAIN 1

/* System matrix: X*^T X (Eq. core_ui, the paper's form, solved by LU with
 * partial pivoting), X*^T X* (symmetric variant, Cholesky), or X^T X (full
 * ALS, Eq. U format, Cholesky). */
#define ALS_GRAM_ASYM 0
#define ALS_GRAM_SYM 1
#define ALS_GRAM_FULL 2

/* Arithmetic of the Gram assembly (the solve is FP32 in every mode):
 *   ALS_FP32    FP32 on CUDA cores for n_f <= 32; for n_f > 32 the
 *               FP32-accurate split TF32 on tensor cores (as ALS_FP32_TC).
 *   ALS_TF32    TF32 inputs, FP32 accumulation, tensor cores (tcgen05).
 *   ALS_BF16    BF16 inputs, FP32 accumulation, tensor cores (tcgen05).
 *   ALS_FP32_TC split TF32 (x = hi + lo, hi*hi + hi*lo + lo*hi accumulated in
 *               FP32) on tensor cores for every n_f.
 * Rows with at most 32 observations and n_f <= 32 are assembled in FP32 on
 * CUDA cores in every mode. */
#define ALS_FP32 0
#define ALS_TF32 1
#define ALS_BF16 2
#define ALS_FP32_TC 3

/* Per-row flags written by the solve. */
/* refine_steps = ALS_REFINE_AUTO: 0 for ALS_FP32 and ALS_FP32_TC, 1 for
 * ALS_TF32, 2 for ALS_BF16 - the steps after which a mixed-precision fit
 * tracks the FP32 one (BF16 rounds to 8 significant bits, TF32 to 11). */
#define ALS_REFINE_AUTO (-1)

/* Sketch of a row's design slice:
 *   ALS_SKETCH_SLICE   Algorithm 2: CES (Algorithm 1) on every row's slice.
 *   ALS_SKETCH_FACTOR  the fast variant of Sec. 3: CES once per half-sweep on
 *                      the whole design factor Y (n_cols rows, the budget
 *                      rule evaluated at n = n_cols, ties to the lower row of
 *                      Y); a row's sketch is that selection restricted to its
 *                      slice, so a row keeps the rate only on average. */
#define ALS_SKETCH_SLICE 0
#define ALS_SKETCH_FACTOR 1

#define ALS_FLAG_RATIO 1     /* pivot ratio above pivot_ratio_max */
#define ALS_FLAG_SINGULAR 2  /* zero / non-positive pivot: the row was set to 0 */
#define ALS_FLAG_FP64 4      /* the row was re-assembled and re-solved in FP64 */

typedef struct als_csr {
    int64_t n_rows;          /* rows of this side (users, or items for R^T) */
    int64_t n_cols;          /* rows of the other side's factor */
    int64_t nnz;
    const int64_t* indptr;   /* device, n_rows + 1, indptr[0] = 0, indptr[n_rows] = nnz */
    const int32_t* indices;  /* device, nnz, in [0, n_cols), ascending within a row */
    const float* values;     /* device, nnz, finite ratings */
} als_csr;

typedef struct als_options {
    int n_f;                 /* rank; 1..128 */
    float lambda;            /* regularisation */
    double budget;           /* CES rate r in [0, 1]; s_i = floor(n_i * r) per column */
    int64_t min_keep;        /* 0 = off; else s_i = min(n_i, max(s_i, min_keep)) */
    int reg_mode;            /* ALS_REG_* */
    int gram_mode;           /* ALS_GRAM_* */
    int precision;           /* ALS_FP32, ALS_TF32, ALS_BF16, ALS_FP32_TC */
    double pivot_ratio_max;  /* flag threshold on max pivot / min pivot, e.g. 1e6 */
    int fp64_fallback;       /* 1: rows flagged by the FP32 solve (ratio above
                                pivot_ratio_max, or a zero pivot) are
                                re-assembled from the data and re-solved in
                                FP64 (flag ALS_FLAG_FP64); 0: off */
    int refine_steps;        /* iterative-refinement steps after the solve (0 to 3,
                                or ALS_REFINE_AUTO): each recomputes the residual
                                of the FP32 system from the data and solves the
                                assembled G again (CTA and split rows) */
    int64_t fixed_keep;      /* 0: the rate rule s_i = floor(n_i r); > 0: the
                                fixed subsample size of Sec. 3, s_i =
                                min(n_i, fixed_keep) per column (budget unused) */
    int sketch;              /* ALS_SKETCH_SLICE or ALS_SKETCH_FACTOR */
} als_options;

typedef struct als_report {
    int64_t rows_flagged;     /* rows with ALS_FLAG_RATIO set, last half-sweep */
    int64_t rows_singular;    /* rows with ALS_FLAG_SINGULAR set, last half-sweep */
    int64_t rows_fp64;        /* rows re-solved in FP64, last half-sweep */
    double max_pivot_ratio;   /* largest pivot ratio seen, last half-sweep */
    double test_rmse;         /* als_fit: test RMSE after the last sweep (NaN if no test set) */
    double objective;         /* als_fit: Eq. (object function) after the last sweep, with the
                                 handle's regulariser mode (NaN from als_get_report) */
    int sweeps_done;
} als_report;

typedef struct als_handle als_handle;

/* Default options: n_f = 32, lambda = 0.05, budget = 0.25, weighted lambda,
 * asymmetric Gram, FP32, pivot_ratio_max = 1e6, FP64 fallback on,
 * refine_steps = ALS_REFINE_AUTO, the rate rule (fixed_keep = 0), the
 * per-slice sketch of Algorithm 2. */
void als_default_options(als_options* opt_host);

/* Create a handle bound to the current CUDA device and to cuda_stream
 * (a cudaStream_t; NULL = the legacy default stream). */
int als_create(als_handle** handle_host, const als_options* opt_host, void* cuda_stream);
int als_destroy(als_handle* h);
int als_set_stream(als_handle* h, void* cuda_stream);
int als_get_options(const als_handle* h, als_options* opt_host);

/* Validate one side's rating structure (sorted unique in-range indices,
 * monotone indptr, finite values) and build its row plan (rows bucketed by
 * length). Synchronises the stream. Later calls with the same indptr
 * pointer, n_rows and nnz reuse the plan; other calls prepare implicitly.
 * Every call that reuses a plan checks the buffers again on the device,
 * without synchronising (also inside a captured graph, on every replay):
 * if their indices or values were refilled with invalid ones, the next call
 * that reads the device error words (als_get_report, als_fit, als_fit_host)
 * returns ALS_ERR_CSR or ALS_ERR_NONFINITE, and the results since the last
 * report are not valid. Kernels clamp out-of-range indices, so such buffers
 * never make a gather read outside the factor. A refilled indptr (changed
 * row structure) must be announced by calling als_prepare again, which
 * re-validates synchronously and rebuilds the plan when the rows changed.
 * Call it once per structure before capturing work into a CUDA graph. */
int als_prepare(als_handle* h, const als_csr* R_side);

/* One half-sweep of Algorithm 2 for the side R_side: for every row i,
 * CES on Y[I_i] and Eq. (core_ui) (or Eq. U format for ALS_GRAM_FULL).
 * Y_in: n_cols x n_f; X_out: n_rows x n_f (rows with n_i = 0 get 0).
 * flags_out (nullable): int32 per row, ALS_FLAG_* bits. Y_in and X_out
 * must not overlap. */
int als_half_sweep(als_handle* h, const als_csr* R_side, const float* Y_in, float* X_out,
                   int32_t* flags_out);

/* CES masks only (Algorithm 1 applied to every row's slice): masks_out holds
 * nnz x ceil(n_f/32) uint32 words in CSR storage order; bit (a mod 32) of
 * word a/32 is set when element (k, a) is kept. */
int als_select(als_handle* h, const als_csr* R_side, const float* Y_in, uint32_t* masks_out);

/* The assembled systems of Eq. (core_ui): G_out n_rows x n_f x n_f (row-major,
 * regulariser already on the diagonal), b_out n_rows x n_f. */
int als_assemble(als_handle* h, const als_csr* R_side, const float* Y_in, float* G_out, float* b_out);

/* Solve n_rows independent systems G x = b (G n_rows x n_f x n_f, b n_rows x
 * n_f) with the handle's method (LU with partial pivoting for ALS_GRAM_ASYM,
 * Cholesky otherwise). flags_out nullable. */
int als_solve(als_handle* h, int64_t n_rows, const float* G, const float* b, float* X_out,
              int32_t* flags_out);

/* Sum of squared errors over n entries (r_e - u_{iu_e} . m_{im_e})^2,
 * accumulated in FP64 in a fixed order; written to sse_host (synchronises). */
int als_eval_sse(als_handle* h, int64_t n, const int32_t* iu, const int32_t* im, const float* r,
                 const float* U, const float* M, double* sse_host);

/* As als_eval_sse, but the FP64 sum is written to sse_dev (one double in
 * device memory) without synchronising. */
int als_eval_sse_async(als_handle* h, int64_t n, const int32_t* iu, const int32_t* im, const float* r,
                       const float* U, const float* M, double* sse_dev);

/* Test-set SSE that allocates nothing: no handle, no cudaMalloc or cudaFree,
 * no allocating library call. The paper has no counterpart; this is for
 * callers that may not allocate device memory when they evaluate:
 *   - code running while its stream is captured into a CUDA graph, where
 *     allocation calls are not allowed;
 *   - programs that give all device memory to their own pool allocator at
 *     start-up and forbid raw allocations afterwards;
 *   - services held to a fixed device-memory budget.
 * Arguments as in als_eval_sse, plus n_f and the stream (a cudaStream_t,
 * NULL = legacy default stream). The FP64 sum is written to sse_dev without
 * synchronising.
 *
 * Scratch: a file-scope device array of ALS_SSE_STATIC_MAX_BLOCKS FP64
 * partial sums (32 KiB). Every GPU that loads the library holds it until the
 * process exits. Each 256-thread block covers up to
 * ALS_SSE_STATIC_ENTRIES_PER_BLOCK entries, so n may not exceed
 * ALS_SSE_STATIC_MAX_ENTRIES (2^26): larger n returns ALS_ERR_ARG and
 * enqueues nothing.
 * The first call on a device looks up the array's device address with that
 * device current, and caches it per (device, CUDA context): a call under a
 * new context (after cudaDeviceReset, for instance) looks it up again. Make
 * the first call in a context before any stream capture.
 * All calls share the one array. A call writes every partial it later reads,
 * so nothing carries over from a previous call. Calls that overlap on the GPU
 * (other streams or threads) race on the array and must be serialised by the
 * caller. */
#define ALS_SSE_STATIC_MAX_BLOCKS 4096
#define ALS_SSE_STATIC_ENTRIES_PER_BLOCK 16384
#define ALS_SSE_STATIC_MAX_ENTRIES ((int64_t)ALS_SSE_STATIC_MAX_BLOCKS * ALS_SSE_STATIC_ENTRIES_PER_BLOCK)
int als_eval_sse_static(int64_t n, const int32_t* iu, const int32_t* im, const float* r, const float* U,
                        const float* M, int n_f, double* sse_dev, void* cuda_stream);

/* Eq. (object function) at (U, M): sum over the training entries of R_users
 * of (r_ij - u_i . m_j)^2 plus lambda (sum_i n_i |u_i|^2 + sum_j n_j |m_j|^2)
 * with the handle's lambda and weighted regulariser (n_i, n_j the row counts
 * of R_users and R_items), or lambda (sum_i |u_i|^2 + sum_j |m_j|^2) with
 * ALS_REG_PLAIN. Products FP32, sums FP64 in a fixed order. Synchronises.
 * Only R_items' indptr is read. */
int als_objective(als_handle* h, const als_csr* R_users, const als_csr* R_items, const float* U, const float* M,
                  double* obj_host);

/* Relative error of Sec. 5.1 over n entries E: sqrt(sum_E (r - u_i . m_j)^2)
 * / sqrt(sum_E r^2) - ReMSE on the empirical (training) set, P-ReMSE on the
 * prediction (missing) set - for one replication. Synchronises; NaN for an
 * empty set. */
int als_eval_remse(als_handle* h, int64_t n, const int32_t* iu, const int32_t* im, const float* r, const float* U,
                   const float* M, double* remse_host);

/* Recommendation metrics of Sec. 5.1. For every user i (row of R_train, the
 * training ratings), the items not rated in R_train are ranked by the FP32
 * predicted rating u_i . m_j (products accumulated by fmaf in feature order;
 * ties: lower item first) and the first K = max(k_hit, k_ndcg) <= 16 are
 * kept (topk_out, nullable: n_u x K int32, -1 when fewer items are unrated).
 * Against each user's relevant items (rel: CSR over the same users, sorted
 * item ids, e.g. held-out items rated at least a threshold): Hit@k_hit is 1
 * when one of the first k_hit items is relevant; NDCG@k_ndcg = DCG / IDCG
 * with binary gains, DCG = sum_p rel_p / log2(p + 2) over positions p =
 * 0..k_ndcg-1, IDCG the same with min(k_ndcg, |rel_i|) relevant items in
 * front. The means over users with at least one relevant item go to
 * hit_host and ndcg_host, their number to n_eval_host (nullable).
 * Synchronises. R_train.n_cols (the items) may be at most 1,500,000. */
int als_eval_ranking(als_handle* h, const als_csr* R_train, const als_csr* rel, const float* U, const float* M,
                     int k_hit, int k_ndcg, int32_t* topk_out, double* hit_host, double* ndcg_host,
                     int64_t* n_eval_host);

/* Kernel timing: while enabled, every kernel the handle launches is
 * bracketed by CUDA events on the handle's stream, and half-sweeps run on
 * that stream alone (no side streams), so each event pair times one launch
 * by itself; results are bit-identical either way. als_kernel_time
 * synchronises and returns the summed event time (ms) and the number of
 * launches of the kernels whose family name is `name` ("cta_rows",
 * "warp_rows", "solve_rows", "sse", ...) since profiling was enabled;
 * name NULL sums every family. Enabling again resets the sums. */
int als_profile(als_handle* h, int enable);
int als_kernel_time(als_handle* h, const char* name, double* ms_host, int64_t* launches_host);

/* Counters of the last half-sweep (synchronises). Returns ALS_ERR_TIMEOUT,
 * with the report still filled, when a bounded device wait ran out since the
 * last report: a tensor-core Gram pipeline that gives up on a completion
 * barrier after 1 s of GPU time stops issuing work, waits once more (bounded)
 * for what it had in flight, frees its tensor memory, stores zero systems and
 * records the timeout in a device error word, which this call reads and
 * clears. After ALS_ERR_TIMEOUT the results of the calls since the last
 * report are undefined; destroy the handle and create a new one before
 * relying on it again. als_fit, als_fit_host and als_batch_fit return it the
 * same way. */
int als_get_report(als_handle* h, als_report* rep_host);

/* Self-test of that mechanism: one thread waits up to limit_ns (0..2e9) of
 * GPU time on a barrier that nothing arrives at and records the timeout like
 * the pipelines do. keep_record 0: the call synchronises, reads and clears
 * the record and returns ALS_ERR_TIMEOUT. keep_record 1: the call only
 * enqueues the wait and returns ALS_OK, leaving the record for the next call
 * that reads it (als_get_report, als_fit, als_fit_host). Nothing faults or
 * hangs. */
int als_wait_selftest(als_handle* h, int64_t limit_ns, int keep_record);

/* One full sweep: users from M (into U), then items from the new U (into M). */
int als_sweep(als_handle* h, const als_csr* R_users, const als_csr* R_items, float* U, float* M);

/* Algorithm 2: `sweeps` sweeps starting from M (in: M^(0), out: result);
 * U is output only. rep_host nullable; when given it gets the counters of
 * the last half-sweep, the objective of Eq. (object function) after the last
 * sweep (als_objective) and, if test entries are given (n_test > 0), the
 * test RMSE. On a created stream, after the first sweep the remaining sweeps
 * replay a CUDA graph of one sweep (captured on the first call with these
 * buffers). The call always ends by synchronising the stream to read the
 * device error word (also when rep_host is NULL), so a bounded device wait
 * that ran out during the fit returns ALS_ERR_TIMEOUT. */
int als_fit(als_handle* h, const als_csr* R_users, const als_csr* R_items, int sweeps,
            float* U, float* M, int64_t n_test, const int32_t* test_u, const int32_t* test_m,
            const float* test_r, als_report* rep_host);

/* als_fit from HOST buffers: copies both sides' CSR arrays, M^(0) and the
 * test entries to the device, fits, and copies U and M back to the host
 * (synchronises). Uses the handle's workspace for device copies. The item
 * side and the test entries go over a copy stream of the handle and the
 * item side is validated there while the first user half-sweep runs; every
 * host buffer is out of use when the call returns, also on error. Plans and
 * the captured sweep tied to the workspace are re-checked on every call. */
int als_fit_host(als_handle* h, int64_t n_u, int64_t n_m, int64_t nnz,
                 const int64_t* user_indptr_host, const int32_t* user_indices_host,
                 const float* user_values_host, const int64_t* item_indptr_host,
                 const int32_t* item_indices_host, const float* item_values_host, int sweeps,
                 float* U_host, float* M_host, int64_t n_test, const int32_t* test_u_host,
                 const int32_t* test_m_host, const float* test_r_host, als_report* rep_host);

/* ---------------------------------------------------------------------------
 * Autotuning of the row schedule on the live problem.
 *
 *   split_at_middle  1: rows longer than the middle CTA capacity take the
 *                    split (multi-CTA) path; 0: only rows longer than the
 *                    largest capacity do.
 *   warp_rows        1: rows with <= 32 observations (n_f <= 32) use the
 *                    fused warp-per-row kernel; 0: the CTA kernel.
 *   tc_gram          ALS_FP32 at n_f <= 32 only - 1: assemble with the
 *                    FP32-accurate split-TF32 tensor-core Gram instead of
 *                    CUDA cores (both meet the same accuracy).
 */
typedef struct als_tuning {
    int split_at_middle;
    int warp_rows;
    int tc_gram;
    double ms_per_sweep;  /* als_autotune: time of the chosen schedule */
} als_tuning;

/* Time every candidate schedule over `trials` sweeps (after one warm-up
 * sweep) on this problem, keep the fastest in the handle and return it. A
 * process-wide cache keyed by (n_f, precision, log2 histogram of both sides'
 * row lengths) skips the timing for a problem of the same shape. U and M
 * are overwritten (M is restored to its value on entry). Synchronises. */
int als_autotune(als_handle* h, const als_csr* R_users, const als_csr* R_items, float* U, float* M, int trials,
                 als_tuning* chosen_host);
/* Set (or read back) the schedule explicitly; plans are rebuilt lazily. */
int als_set_tuning(als_handle* h, const als_tuning* t_host);
int als_get_tuning(const als_handle* h, als_tuning* t_host);

/* ---------------------------------------------------------------------------
 * Batches of independent completion problems.
 *
 * Problems with the same n_f are concatenated block-diagonally on the device
 * (user and item indices shifted by each problem's offsets), so one set of
 * launches per half-sweep serves every problem of that width; rows never
 * interact, so each problem's result equals the one it gets alone. One
 * sweep of all groups is captured into a CUDA graph and replayed. Options
 * other than n_f come from opt; cuda_stream must not be the legacy default
 * stream (graph capture needs a created stream). The fast variant
 * (ALS_SKETCH_FACTOR) is not built for batches: ALS_ERR_UNSUPPORTED. */
typedef struct als_problem {
    als_csr users;  /* R in CSR (device arrays) */
    als_csr items;  /* R^T in CSR (device arrays) */
    int n_f;
    float* U;       /* device, users.n_rows x n_f: output */
    float* M;       /* device, items.n_rows x n_f: in M^(0), out result */
} als_problem;

typedef struct als_batch als_batch;

/* Build the groups, their row plans and the captured sweep (synchronises).
 * The problems' arrays must stay valid until als_batch_destroy. */
int als_batch_create(als_batch** batch_host, const als_options* opt_host, int n_problems,
                     const als_problem* problems_host, void* cuda_stream);
/* `sweeps` sweeps of Algorithm 2 for every problem from its M (read at the
 * start), writing U and M back. Enqueued on the batch stream; the call then
 * synchronises it to read every width group's device error word and returns
 * ALS_ERR_TIMEOUT if a bounded device wait ran out in any group. */
int als_batch_fit(als_batch* b, int sweeps);
/* CES masks (as als_select) of one side (0 users, 1 items) of problem
 * `problem`, computed on the batch's block-diagonal structure with that
 * problem's design factor Y (device, the other side's rows x n_f; copied into
 * the batch's factor buffer, which the next als_batch_fit overwrites).
 * masks_out: the problem's nnz x ceil(n_f/32) words in its own CSR order.
 * Synchronises. */
int als_batch_select(als_batch* b, int problem, int side, const float* Y, uint32_t* masks_out);
/* Kernel launches in one replayed sweep (all groups). */
int64_t als_batch_launches_per_sweep(const als_batch* b);
int als_batch_destroy(als_batch* b);

/* ---------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper).
 *
 * Per-row features of one side from the other side's factor Y:
 *   feat_i = [ sum_j r_ij y_j / sum_j r_ij  (n_f values),  log(1 + n_i),
 *              mean_j r_ij ]                         (n_rows x (n_f + 2))
 * and a 3-layer MLP  y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3  (GELU with
 * erf) trained on MSE by Adam (beta 0.9 / 0.999, eps 1e-8). Master weights
 * are FP32; the forward and backward products use their BF16 rounding;
 * activations and sums are FP32 and every reduction has a fixed order. The
 * products run on the tensor cores (tcgen05 kind::tf32; BF16 weights are
 * exact in TF32, FP32 operands are split into TF32 hi + lo parts). A bounded
 * tensor-core wait that runs out is returned as ALS_ERR_TIMEOUT by the next
 * call of the network that synchronises (grad, train_step with a loss,
 * get_params).
 * Parameters (FP32, flat): W1 (hidden x in), b1, W2 (hidden x hidden), b2,
 * W3 (out x hidden), b3. X, Y, T are device arrays, row-major. */
typedef struct als_mlp als_mlp;
int als_features(const als_csr* R_side, const float* Y, int n_f, float* feat_out, void* cuda_stream);
/* Weights uniform in +-1/sqrt(fan_in) from SplitMix64(seed), zero biases. */
int als_mlp_create(als_mlp** mlp_host, int in_dim, int hidden, int out_dim, uint64_t seed, void* cuda_stream);
int als_mlp_destroy(als_mlp* m);
int64_t als_mlp_num_params(const als_mlp* m);
int als_mlp_set_params(als_mlp* m, const float* params_host);  /* also resets Adam state (synchronises) */
int als_mlp_get_params(als_mlp* m, float* params_host);        /* synchronises */
int als_mlp_forward(als_mlp* m, int64_t n, const float* X, float* Y);
/* Gradient of the mean squared error at the current weights (no update);
 * grads_host (nullable) gets n_params floats; synchronises. */
int als_mlp_grad(als_mlp* m, int64_t n, const float* X, const float* T, float* grads_host, double* loss_host);
/* One Adam step on a batch of n rows; loss_host (nullable) gets the batch
 * loss before the step (synchronises only when given). */
int als_mlp_train_step(als_mlp* m, int64_t n, const float* X, const float* T, float lr, double* loss_host);

/* ---------------------------------------------------------------------------
 * Roofline probes (no counterpart in the paper: the measured peaks that the
 * kernels' roofline fractions are taken against). Each allocates and frees
 * its own buffers, runs one warm-up and one timed launch on cuda_stream
 * (a cudaStream_t, NULL = legacy default stream), synchronises, and writes
 * the achieved rate to value_host (TFLOP/s, or GB/s for the two memory
 * probes) and the timed launch's CUDA-event duration to ms_host (nullable):
 *   ALS_PROBE_FFMA       FP32 FMA, 8 independent chains per thread
 *   ALS_PROBE_DFMA       FP64 FMA, the same shape
 *   ALS_PROBE_TC_BF16    tcgen05.mma kind::f16 (BF16), M 128 x N 256, one CTA
 *                        per SM, operands in shared memory, accumulator in TMEM
 *   ALS_PROBE_TC_TF32    the same with kind::tf32
 *   ALS_PROBE_L2_GATHER  random 128-byte row gathers from a 16 MB factor
 *   ALS_PROBE_HBM_COPY   a 2 GB device-to-device copy kernel (read + write)
 * ALS_ERR_TIMEOUT when a tensor-core probe's bounded wait ran out. */
#define ALS_PROBE_FFMA 0
#define ALS_PROBE_DFMA 1
#define ALS_PROBE_TC_BF16 2
#define ALS_PROBE_TC_TF32 3
#define ALS_PROBE_L2_GATHER 4
#define ALS_PROBE_HBM_COPY 5
int als_probe(int kind, double* value_host, double* ms_host, void* cuda_stream);

/* Bytes of device workspace the handle currently holds. */
int64_t als_workspace_bytes(const als_handle* h);

/* Number of kernel launches the handle has enqueued since creation. */
int64_t als_launch_count(const als_handle* h);

const char* als_status_string(int status);
const char* als_last_error(const als_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* CORE_ALS_H */
