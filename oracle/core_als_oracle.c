/*
 * FP64 CPU oracle for core-elements ALS (Core-ALS).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA path is checked against. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it. It shares no code, header or constant
 * with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, following the paper step by step:
 *
 *   Algorithm 1 (CES): for every column a of a design slice X (n x f), keep
 *     the s largest |x_ka| and zero the rest. Here s = floor(n * r) (the
 *     per-slice rule of Sec. 3: "floor(|I_i| * r) elements with the largest
 *     absolute values in each column"). Ties in |x| go to the lower position
 *     k, where position is the order of the row's sorted index list.
 *
 *   Eq. (core_ui) / (core_mj): with X* = S (.) X,
 *       x_i = (X*^T X + lambda n_i E)^{-1} X*^T r_i         (asymmetric form)
 *     and, as an option, the symmetric variant with X*^T X* in place of
 *     X*^T X. n_i is the full number of observations of the row (the
 *     weighted-lambda regulariser of Eq. (object function)); the PLAIN
 *     regulariser mode uses lambda alone.
 *
 *   Eq. (U format) / (M format): full ALS, the same estimator with S = all
 *     ones; solved by Cholesky because the matrix is symmetric positive
 *     definite for lambda > 0.
 *
 *   Budget: s = floor(n * r) per column, or the fixed subsample size
 *     s = min(n, fixed_keep) (the fixed-size version of Sec. 3).
 *
 *   Fast variant (Sec. 3): CES applied once per half-sweep to the whole
 *     design factor, each row's sketch being that selection restricted to
 *     its slice.
 *
 *   Eq. (object function): f(U, M) = sum_I (r_ij - u_i m_j^T)^2
 *       + lambda (sum_i n_ui |u_i|^2 + sum_j n_mj |m_j|^2).
 *
 *   Sec. 5.1 evaluation: ReMSE / P-ReMSE (relative root sum of squares over
 *     the empirical and the prediction set), and the recommendation metrics
 *     Hit@k and NDCG@k over ranked lists of unrated items.
 *
 * Linear solves: Gaussian elimination with partial pivoting for the
 * asymmetric system (the paper only assumes it is of full rank), Cholesky for
 * the symmetric ones. Pivot ratio = max pivot / min pivot, with pivot |U_kk|
 * for LU and L_kk^2 for Cholesky; a row whose ratio exceeds the threshold, or
 * whose pivot is zero or not positive, is flagged. A row whose factorisation
 * breaks down gets x_i = 0.
 *
 * Every loop runs in the order the definitions are written; rows are
 * independent and are spread over OpenMP threads when the library is built
 * with -fopenmp (each row's arithmetic is unchanged by that).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_REG_WEIGHTED = 0, OR_REG_PLAIN = 1 };
enum { OR_GRAM_ASYM = 0, OR_GRAM_SYM = 1, OR_GRAM_FULL = 2 };
enum { OR_FLAG_RATIO = 1, OR_FLAG_SINGULAR = 2 };

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Elements kept per column of an n-row slice.
 *   rate rule (fixed_keep == 0): s = floor(n * r) in IEEE double (Sec. 3);
 *   fixed subsample size (fixed_keep > 0): s = min(n, fixed_keep), the
 *     version with a fixed subsample size mentioned in Sec. 3;
 * then raised to min(n, min_keep) when min_keep > 0.
 */
int64_t oracle_budget(int64_t n, double r, int64_t min_keep, int64_t fixed_keep) {
    int64_t s;
    if (fixed_keep > 0) {
        s = fixed_keep < n ? fixed_keep : n;
    } else {
        double p = (double)n * r;
        s = (int64_t)floor(p);
    }
    if (s > n) s = n;
    if (s < 0) s = 0;
    if (min_keep > 0 && s < min_keep) s = (min_keep < n) ? min_keep : n;
    return s;
}

typedef struct { double mag; int64_t pos; } or_item;

/* Larger |x| first; equal |x| -> lower position first. */
static int or_cmp(const void* pa, const void* pb) {
    const or_item* a = (const or_item*)pa;
    const or_item* b = (const or_item*)pb;
    if (a->mag > b->mag) return -1;
    if (a->mag < b->mag) return 1;
    if (a->pos < b->pos) return -1;
    if (a->pos > b->pos) return 1;
    return 0;
}

/*
 * Algorithm 1 (CES) on one slice. X is n x f row-major. keep[k*f + a] = 1 when
 * element (k, a) is in the sketch. items is scratch of n entries.
 */
void oracle_ces(int64_t n, int f, const double* X, int64_t s, uint8_t* keep, or_item* items) {
    memset(keep, 0, (size_t)(n * f));
    for (int a = 0; a < f; ++a) {
        for (int64_t k = 0; k < n; ++k) {
            items[k].mag = fabs(X[k * f + a]);
            items[k].pos = k;
        }
        qsort(items, (size_t)n, sizeof(or_item), or_cmp);
        for (int64_t q = 0; q < s && q < n; ++q) keep[items[q].pos * f + a] = 1;
    }
}

/*
 * Fast variant of Core-ALS (Sec. 3): CES is applied once, before the
 * half-sweep, to the whole design factor Y (n_other x f) instead of to every
 * row's slice. keep_Y (n_other x f) marks, per column, the s = budget(n_other)
 * entries of largest |y_ja| (ties to the lower row j). A row's sketch is this
 * selection restricted to its slice: X*_ka = keep_Y[I_i[k]][a] x_ka, so the
 * number kept in a row's column only follows the rate on average.
 * Returns 0, or -1 when scratch memory could not be allocated.
 */
int oracle_factor_sketch(int64_t n_other, int f, const double* Y, double budget, int64_t min_keep,
                         int64_t fixed_keep, uint8_t* keep_Y) {
    or_item* items = (or_item*)malloc((size_t)(n_other > 0 ? n_other : 1) * sizeof(or_item));
    if (!items) return -1;
    oracle_ces(n_other, f, Y, oracle_budget(n_other, budget, min_keep, fixed_keep), keep_Y, items);
    free(items);
    return 0;
}

/* The keep pattern of a row's slice: from its own CES (keep_Y == NULL) or
 * from the factor-wide selection of the fast variant. */
static void or_row_keep(int64_t lo, int64_t n, int f, const int32_t* indices, const double* X, int64_t s,
                        const uint8_t* keep_Y, uint8_t* keep, or_item* items) {
    if (keep_Y == NULL) {
        oracle_ces(n, f, X, s, keep, items);
        return;
    }
    for (int64_t k = 0; k < n; ++k)
        for (int a = 0; a < f; ++a) keep[k * f + a] = keep_Y[(int64_t)indices[lo + k] * f + a];
}

/*
 * Normal equations of one row. G is f x f row-major, b has f entries.
 *   ASYM: G[a][c] = sum_k keep(k,a) x_ka x_kc,       b[a] = sum_k keep(k,a) x_ka r_k
 *   SYM : G[a][c] = sum_k keep(k,a) keep(k,c) x_ka x_kc, b as ASYM
 *   FULL: keep = 1 everywhere.
 * Then G[a][a] += reg.
 */
void oracle_assemble(int64_t n, int f, const double* X, const double* r, const uint8_t* keep,
                     int gram_mode, double reg, double* G, double* b) {
    for (int a = 0; a < f; ++a) {
        for (int c = 0; c < f; ++c) {
            double acc = 0.0;
            for (int64_t k = 0; k < n; ++k) {
                double wa = (gram_mode == OR_GRAM_FULL) ? 1.0 : (double)keep[k * f + a];
                double wc = (gram_mode == OR_GRAM_SYM) ? (double)keep[k * f + c] : 1.0;
                acc += wa * X[k * f + a] * wc * X[k * f + c];
            }
            G[a * f + c] = acc;
        }
        double acc = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            double wa = (gram_mode == OR_GRAM_FULL) ? 1.0 : (double)keep[k * f + a];
            acc += wa * X[k * f + a] * r[k];
        }
        b[a] = acc;
        G[a * f + a] += reg;
    }
}

/*
 * Gaussian elimination with partial pivoting on A (f x f, overwritten) and
 * right-hand side rhs (overwritten), solution in x. Returns flags and the
 * pivot ratio max|U_kk| / min|U_kk|.
 */
int oracle_solve_lu(int f, double* A, double* rhs, double* x, double ratio_max, double* ratio_out) {
    double pmax = 0.0, pmin = INFINITY;
    int flags = 0;
    for (int k = 0; k < f; ++k) {
        int p = k;
        double best = fabs(A[k * f + k]);
        for (int i = k + 1; i < f; ++i) {
            double v = fabs(A[i * f + k]);
            if (v > best) { best = v; p = i; }
        }
        if (best == 0.0) {
            for (int j = 0; j < f; ++j) x[j] = 0.0;
            if (ratio_out) *ratio_out = INFINITY;
            return OR_FLAG_SINGULAR | OR_FLAG_RATIO;
        }
        if (p != k) {
            for (int j = 0; j < f; ++j) {
                double t = A[k * f + j]; A[k * f + j] = A[p * f + j]; A[p * f + j] = t;
            }
            double t = rhs[k]; rhs[k] = rhs[p]; rhs[p] = t;
        }
        if (best > pmax) pmax = best;
        if (best < pmin) pmin = best;
        for (int i = k + 1; i < f; ++i) {
            double l = A[i * f + k] / A[k * f + k];
            A[i * f + k] = 0.0;
            for (int j = k + 1; j < f; ++j) A[i * f + j] -= l * A[k * f + j];
            rhs[i] -= l * rhs[k];
        }
    }
    for (int k = f - 1; k >= 0; --k) {
        double acc = rhs[k];
        for (int j = k + 1; j < f; ++j) acc -= A[k * f + j] * x[j];
        x[k] = acc / A[k * f + k];
    }
    double ratio = pmax / pmin;
    if (ratio_out) *ratio_out = ratio;
    if (ratio > ratio_max) flags |= OR_FLAG_RATIO;
    return flags;
}

/*
 * Cholesky A = L L^T (lower triangle of A used, A overwritten by L), then
 * L y = rhs and L^T x = y. Pivot ratio max L_kk^2 / min L_kk^2.
 */
int oracle_solve_chol(int f, double* A, double* rhs, double* x, double ratio_max, double* ratio_out) {
    double pmax = 0.0, pmin = INFINITY;
    for (int k = 0; k < f; ++k) {
        double d = A[k * f + k];
        for (int j = 0; j < k; ++j) d -= A[k * f + j] * A[k * f + j];
        if (!(d > 0.0)) {
            for (int j = 0; j < f; ++j) x[j] = 0.0;
            if (ratio_out) *ratio_out = INFINITY;
            return OR_FLAG_SINGULAR | OR_FLAG_RATIO;
        }
        if (d > pmax) pmax = d;
        if (d < pmin) pmin = d;
        double lkk = sqrt(d);
        A[k * f + k] = lkk;
        for (int i = k + 1; i < f; ++i) {
            double v = A[i * f + k];
            for (int j = 0; j < k; ++j) v -= A[i * f + j] * A[k * f + j];
            A[i * f + k] = v / lkk;
        }
    }
    for (int i = 0; i < f; ++i) {
        double v = rhs[i];
        for (int j = 0; j < i; ++j) v -= A[i * f + j] * x[j];
        x[i] = v / A[i * f + i];
    }
    for (int i = f - 1; i >= 0; --i) {
        double v = x[i];
        for (int j = i + 1; j < f; ++j) v -= A[j * f + i] * x[j];
        x[i] = v / A[i * f + i];
    }
    double ratio = pmax / pmin;
    if (ratio_out) *ratio_out = ratio;
    return ratio > ratio_max ? OR_FLAG_RATIO : 0;
}

typedef struct {
    double* X; double* r; uint8_t* keep; or_item* items; double* G; double* b; double* x;
} or_scratch;

static int or_scratch_alloc(or_scratch* s, int64_t nmax, int f) {
    size_t n = (size_t)(nmax > 0 ? nmax : 1);
    s->X = (double*)malloc(n * (size_t)f * sizeof(double));
    s->r = (double*)malloc(n * sizeof(double));
    s->keep = (uint8_t*)malloc(n * (size_t)f);
    s->items = (or_item*)malloc(n * sizeof(or_item));
    s->G = (double*)malloc((size_t)f * (size_t)f * sizeof(double));
    s->b = (double*)malloc((size_t)f * sizeof(double));
    s->x = (double*)malloc((size_t)f * sizeof(double));
    return s->X && s->r && s->keep && s->items && s->G && s->b && s->x;
}

static void or_scratch_free(or_scratch* s) {
    free(s->X); free(s->r); free(s->keep); free(s->items); free(s->G); free(s->b); free(s->x);
}

/* Gather X = Y[I_i] (rows in the order of the row's index list) and r. */
static void or_gather(int64_t lo, int64_t n, const int32_t* indices, const float* values,
                      int f, const double* Y, double* X, double* r) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = indices[lo + k];
        for (int a = 0; a < f; ++a) X[k * f + a] = Y[j * f + a];
        r[k] = (double)values[lo + k];
    }
}

static double or_reg(int reg_mode, double lambda, int64_t n) {
    return reg_mode == OR_REG_PLAIN ? lambda : lambda * (double)n;
}

static int64_t or_max_len(int64_t n_rows, const int64_t* indptr, const int64_t* rows) {
    int64_t m = 0;
    for (int64_t q = 0; q < n_rows; ++q) {
        int64_t i = rows ? rows[q] : q;
        int64_t len = indptr[i + 1] - indptr[i];
        if (len > m) m = len;
    }
    return m;
}

/*
 * One half-sweep of Algorithm 2 (all users, or all items): for each listed
 * row i, CES on its design slice, then Eq. (core_ui) (or the full update when
 * gram_mode is FULL). keep_Y (n_other x f, or NULL) is the factor-wide selection
 * of the fast variant (oracle_factor_sketch); NULL means the per-slice CES of
 * Algorithm 2. Y is the other side's factor (n_other x f); X_out rows
 * i are written (X_out is n_rows_total x f). rows == NULL means every row
 * 0..n_rows-1; otherwise n_rows entries of rows give the subset.
 * flags_out / ratio_out (optional) are indexed like X_out.
 * Returns 0, or -1 when scratch memory could not be allocated.
 */
int oracle_half_sweep(int64_t n_rows, const int64_t* rows, const int64_t* indptr,
                      const int32_t* indices, const float* values, int f, const double* Y,
                      double lambda, double budget, int64_t min_keep, int64_t fixed_keep, int reg_mode,
                      int gram_mode, double ratio_max, const uint8_t* keep_Y, double* X_out,
                      int32_t* flags_out, double* ratio_out) {
    int64_t nmax = or_max_len(n_rows, indptr, rows);
    int err = 0;
#pragma omp parallel
    {
        or_scratch s;
        int ok = or_scratch_alloc(&s, nmax, f);
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < n_rows; ++q) {
            if (!ok) continue;
            int64_t i = rows ? rows[q] : q;
            int64_t lo = indptr[i], n = indptr[i + 1] - indptr[i];
            or_gather(lo, n, indices, values, f, Y, s.X, s.r);
            int64_t sz = (gram_mode == OR_GRAM_FULL) ? n : oracle_budget(n, budget, min_keep, fixed_keep);
            if (gram_mode != OR_GRAM_FULL) or_row_keep(lo, n, f, indices, s.X, sz, keep_Y, s.keep, s.items);
            oracle_assemble(n, f, s.X, s.r, s.keep, gram_mode, or_reg(reg_mode, lambda, n), s.G, s.b);
            double ratio = 0.0;
            int fl = (gram_mode == OR_GRAM_ASYM)
                         ? oracle_solve_lu(f, s.G, s.b, s.x, ratio_max, &ratio)
                         : oracle_solve_chol(f, s.G, s.b, s.x, ratio_max, &ratio);
            for (int a = 0; a < f; ++a) X_out[i * f + a] = s.x[a];
            if (flags_out) flags_out[i] = fl;
            if (ratio_out) ratio_out[i] = ratio;
        }
        or_scratch_free(&s);
    }
    return err ? -1 : 0;
}

/*
 * CES masks of a whole half-sweep, packed as the GPU exports them: for entry
 * e of the CSR (in storage order) word w holds bit (a mod 32) for column
 * a = 32 w + bit. masks has nnz * ceil(f/32) words.
 */
int oracle_select_half(int64_t n_rows, const int64_t* indptr, const int32_t* indices, int f,
                       const double* Y, double budget, int64_t min_keep, int64_t fixed_keep,
                       const uint8_t* keep_Y, uint32_t* masks) {
    int64_t nmax = or_max_len(n_rows, indptr, NULL);
    int words = (f + 31) / 32;
    int err = 0;
#pragma omp parallel
    {
        or_scratch s;
        int ok = or_scratch_alloc(&s, nmax, f);
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n_rows; ++i) {
            if (!ok) continue;
            int64_t lo = indptr[i], n = indptr[i + 1] - indptr[i];
            for (int64_t k = 0; k < n; ++k)
                for (int a = 0; a < f; ++a) s.X[k * f + a] = Y[(int64_t)indices[lo + k] * f + a];
            or_row_keep(lo, n, f, indices, s.X, oracle_budget(n, budget, min_keep, fixed_keep), keep_Y, s.keep,
                        s.items);
            for (int64_t k = 0; k < n; ++k) {
                for (int w = 0; w < words; ++w) {
                    uint32_t m = 0;
                    for (int bit = 0; bit < 32; ++bit) {
                        int a = 32 * w + bit;
                        if (a < f && s.keep[k * f + a]) m |= (uint32_t)1u << bit;
                    }
                    masks[(lo + k) * words + w] = m;
                }
            }
        }
        or_scratch_free(&s);
    }
    return err ? -1 : 0;
}

/* Assembled systems of every row: G is n_rows x f x f, b is n_rows x f. */
int oracle_assemble_half(int64_t n_rows, const int64_t* indptr, const int32_t* indices,
                         const float* values, int f, const double* Y, double lambda, double budget,
                         int64_t min_keep, int64_t fixed_keep, int reg_mode, int gram_mode,
                         const uint8_t* keep_Y, double* G, double* b) {
    int64_t nmax = or_max_len(n_rows, indptr, NULL);
    int err = 0;
#pragma omp parallel
    {
        or_scratch s;
        int ok = or_scratch_alloc(&s, nmax, f);
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n_rows; ++i) {
            if (!ok) continue;
            int64_t lo = indptr[i], n = indptr[i + 1] - indptr[i];
            or_gather(lo, n, indices, values, f, Y, s.X, s.r);
            if (gram_mode != OR_GRAM_FULL)
                or_row_keep(lo, n, f, indices, s.X, oracle_budget(n, budget, min_keep, fixed_keep), keep_Y,
                            s.keep, s.items);
            oracle_assemble(n, f, s.X, s.r, s.keep, gram_mode, or_reg(reg_mode, lambda, n),
                            G + i * (int64_t)f * f, b + i * (int64_t)f);
        }
        or_scratch_free(&s);
    }
    return err ? -1 : 0;
}

/* Solve n_rows independent systems (G, b as above). method 0 = LU, 1 = Cholesky. */
void oracle_solve_batch(int64_t n_rows, int f, const double* G, const double* b, int method,
                        double ratio_max, double* X, int32_t* flags, double* ratios) {
#pragma omp parallel
    {
        double* A = (double*)malloc((size_t)f * f * sizeof(double));
        double* rhs = (double*)malloc((size_t)f * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n_rows; ++i) {
            memcpy(A, G + i * (int64_t)f * f, (size_t)f * f * sizeof(double));
            memcpy(rhs, b + i * (int64_t)f, (size_t)f * sizeof(double));
            double ratio = 0.0;
            int fl = method == 0 ? oracle_solve_lu(f, A, rhs, X + i * (int64_t)f, ratio_max, &ratio)
                                 : oracle_solve_chol(f, A, rhs, X + i * (int64_t)f, ratio_max, &ratio);
            if (flags) flags[i] = fl;
            if (ratios) ratios[i] = ratio;
        }
        free(A);
        free(rhs);
    }
}

/* Sum over listed entries of (r - u_i . m_j)^2 (the data term of Eq. object function). */
double oracle_sse(int64_t n, const int32_t* iu, const int32_t* im, const float* r, int f,
                  const double* U, const double* M) {
    double total = 0.0;
    for (int64_t e = 0; e < n; ++e) {
        double d = (double)r[e];
        for (int a = 0; a < f; ++a) d -= U[(int64_t)iu[e] * f + a] * M[(int64_t)im[e] * f + a];
        total += d * d;
    }
    return total;
}

/* Penalty of one side in Eq. (object function): lambda * sum_i n_i |x_i|^2
 * (weighted lambda), or lambda * sum_i |x_i|^2 for the plain regulariser. */
double oracle_reg_term(int64_t n_rows, const int64_t* indptr, int f, const double* X, double lambda,
                       int reg_mode) {
    double total = 0.0;
    for (int64_t i = 0; i < n_rows; ++i) {
        double sq = 0.0;
        for (int a = 0; a < f; ++a) sq += X[i * f + a] * X[i * f + a];
        total += (reg_mode == OR_REG_PLAIN ? 1.0 : (double)(indptr[i + 1] - indptr[i])) * sq;
    }
    return lambda * total;
}

/*
 * Relative error of Sec. 5.1 over a set of entries E (the empirical set I for
 * ReMSE, the prediction set I^c for P-ReMSE):
 *   sqrt(sum_E (r_ij - u_i . m_j)^2) / sqrt(sum_E r_ij^2)      (one replication).
 * Returns NaN when E is empty or every r_ij is zero.
 */
double oracle_remse(int64_t n, const int32_t* iu, const int32_t* im, const float* r, int f, const double* U,
                    const double* M) {
    double num = 0.0, den = 0.0;
    for (int64_t e = 0; e < n; ++e) {
        double d = (double)r[e];
        for (int a = 0; a < f; ++a) d -= U[(int64_t)iu[e] * f + a] * M[(int64_t)im[e] * f + a];
        num += d * d;
        den += (double)r[e] * (double)r[e];
    }
    return (den > 0.0) ? sqrt(num) / sqrt(den) : NAN;
}

/*
 * Recommendation lists of Sec. 5.1: for every user i, the K items not rated
 * in the training set with the largest predicted rating u_i . m_j, in order
 * (ties: lower item index first). The predicted rating is the FP32 chain
 * acc = fmaf(u_ia, m_ja, acc) for a = 0..f-1 from acc = 0, the precision in
 * which the GPU ranks, so that both sides rank the same numbers. topk is
 * n_u x K item indices, -1 where fewer than K items are unrated.
 */
typedef struct { float score; int32_t item; } or_cand;

static int or_cand_cmp(const void* pa, const void* pb) {
    const or_cand* a = (const or_cand*)pa;
    const or_cand* b = (const or_cand*)pb;
    if (a->score > b->score) return -1;
    if (a->score < b->score) return 1;
    return (a->item < b->item) ? -1 : (a->item > b->item);
}

int oracle_rank_topk(int64_t n_u, int64_t n_m, int f, const float* U, const float* M, const int64_t* train_indptr,
                     const int32_t* train_indices, int K, int32_t* topk) {
    int err = 0;
#pragma omp parallel
    {
        or_cand* c = (or_cand*)malloc((size_t)(n_m > 0 ? n_m : 1) * sizeof(or_cand));
        if (!c) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n_u; ++i) {
            if (!c) continue;
            int64_t q = train_indptr[i], q_end = train_indptr[i + 1], nc = 0;
            for (int64_t j = 0; j < n_m; ++j) {
                while (q < q_end && train_indices[q] < j) ++q;
                if (q < q_end && train_indices[q] == j) continue;  /* rated in training */
                float acc = 0.0f;
                for (int a = 0; a < f; ++a) acc = fmaf(U[i * f + a], M[j * f + a], acc);
                c[nc].score = acc;
                c[nc].item = (int32_t)j;
                ++nc;
            }
            qsort(c, (size_t)nc, sizeof(or_cand), or_cand_cmp);
            for (int p = 0; p < K; ++p) topk[i * K + p] = (p < nc) ? c[p].item : -1;
        }
        free(c);
    }
    return err ? -1 : 0;
}

/*
 * Hit@k_hit and NDCG@k_ndcg (Sec. 5.1) of the lists topk (n_u x K, K >= both
 * k) against each user's relevant items rel (CSR, sorted): for a user with at
 * least one relevant item, hit = 1 when one of the first k_hit listed items
 * is relevant; NDCG = DCG / IDCG with binary gains, DCG = sum over the first
 * k_ndcg positions p (from 0) of rel / log2(p + 2), IDCG the same sum for
 * min(k_ndcg, |rel_i|) relevant items in front. Users without relevant items
 * are skipped; the means are over the others (n_eval of them).
 */
void oracle_rank_metrics(int64_t n_u, const int32_t* topk, int K, int k_hit, int k_ndcg, const int64_t* rel_indptr,
                         const int32_t* rel_indices, double* hit_out, double* ndcg_out, int64_t* n_eval_out) {
    double hit = 0.0, ndcg = 0.0;
    int64_t n_eval = 0;
    for (int64_t i = 0; i < n_u; ++i) {
        int64_t lo = rel_indptr[i], hi = rel_indptr[i + 1];
        if (hi == lo) continue;
        ++n_eval;
        double h = 0.0, dcg = 0.0, idcg = 0.0;
        for (int p = 0; p < K; ++p) {
            int32_t j = topk[i * K + p];
            int is_rel = 0;
            for (int64_t q = lo; q < hi && j >= 0; ++q)
                if (rel_indices[q] == j) is_rel = 1;
            if (p < k_hit && is_rel) h = 1.0;
            if (p < k_ndcg && is_rel) dcg += 1.0 / log2((double)p + 2.0);
        }
        for (int p = 0; p < k_ndcg && p < hi - lo; ++p) idcg += 1.0 / log2((double)p + 2.0);
        hit += h;
        ndcg += dcg / idcg;
    }
    *hit_out = n_eval ? hit / (double)n_eval : NAN;
    *ndcg_out = n_eval ? ndcg / (double)n_eval : NAN;
    *n_eval_out = n_eval;
}
