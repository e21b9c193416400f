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
 *   Eq. (object function): f(U, M) = sum_I (r_ij - u_i m_j^T)^2
 *       + lambda (sum_i n_ui |u_i|^2 + sum_j n_mj |m_j|^2).
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

/* s = floor(n * r) in IEEE double, clamped into [min_keep, n] when min_keep > 0. */
int64_t oracle_budget(int64_t n, double r, int64_t min_keep) {
    double p = (double)n * r;
    int64_t s = (int64_t)floor(p);
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
 * gram_mode is FULL). Y is the other side's factor (n_other x f); X_out rows
 * i are written (X_out is n_rows_total x f). rows == NULL means every row
 * 0..n_rows-1; otherwise n_rows entries of rows give the subset.
 * flags_out / ratio_out (optional) are indexed like X_out.
 * Returns 0, or -1 when scratch memory could not be allocated.
 */
int oracle_half_sweep(int64_t n_rows, const int64_t* rows, const int64_t* indptr,
                      const int32_t* indices, const float* values, int f, const double* Y,
                      double lambda, double budget, int64_t min_keep, int reg_mode, int gram_mode,
                      double ratio_max, double* X_out, int32_t* flags_out, double* ratio_out) {
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
            int64_t sz = (gram_mode == OR_GRAM_FULL) ? n : oracle_budget(n, budget, min_keep);
            if (gram_mode != OR_GRAM_FULL) oracle_ces(n, f, s.X, sz, s.keep, s.items);
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
                       const double* Y, double budget, int64_t min_keep, uint32_t* masks) {
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
            oracle_ces(n, f, s.X, oracle_budget(n, budget, min_keep), s.keep, s.items);
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
                         int64_t min_keep, int reg_mode, int gram_mode, double* G, double* b) {
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
                oracle_ces(n, f, s.X, oracle_budget(n, budget, min_keep), s.keep, s.items);
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

/* lambda * sum_i n_i |x_i|^2 over the rows of one side (weighted-lambda term). */
double oracle_reg_term(int64_t n_rows, const int64_t* indptr, int f, const double* X, double lambda) {
    double total = 0.0;
    for (int64_t i = 0; i < n_rows; ++i) {
        double sq = 0.0;
        for (int a = 0; a < f; ++a) sq += X[i * f + a] * X[i * f + a];
        total += (double)(indptr[i + 1] - indptr[i]) * sq;
    }
    return lambda * total;
}
