/*
 * cv_oracle.c -- CPU oracle for partition-based cross-validation products.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load this file.  The CUDA
 * library never includes, links or calls it, and it uses nothing of the
 * CUDA library.
 *
 * Written from Engstrom & Jensen, "Fast Partition-Based Cross-Validation With
 * Centering and Scaling for X^T X and X^T Y" (arXiv 2401.13185):
 *
 *   cvo_validation_partitions  Algorithm 1 (Definition 1, Lemma 1).
 *   cvo_naive                  Algorithms 2, 4 and 6, generalised to all 16
 *                              centering/scaling combinations (Section 6,
 *                              Table 1).  This is the plain definition
 *                              (Definitions 2-5): for each fold, slice the
 *                              training rows, take their means and standard
 *                              deviations, preprocess, multiply.
 *   cvo_naive_subset           cvo_naive restricted to a list of folds.
 *   cvo_naive_entry            One entry of cvo_naive's output, computed by
 *                              the same arithmetic in the same order (so it
 *                              is bitwise equal to the full computation).
 *   cvo_fast                   Algorithms 3, 5 and 7, generalised the same
 *                              way: products, sums and sums of squares over
 *                              all rows once, then per fold remove the
 *                              validation rows' contribution (Lemmas 2, 3,
 *                              7, 8, 12-14; Propositions 7, 8, 15, 16).
 *   cvo_ridge                  Per-fold ridge / OLS coefficients from the
 *                              products through the normal equations
 *                              (Section 1 names RR and OLS as consumers),
 *                              by Cholesky factorisation.
 *   cvo_press                  The per-fold models' squared prediction error
 *                              on each validation partition (Section 1).
 *
 * Conventions (readings of points the paper leaves open):
 *   - Folds are 0-based: fold f here is partition p = f + 1 of Definition 1.
 *   - ddof in {0, 1}: the standard deviation divides by |T| - ddof.
 *     Definition 4 is the ddof = 1 case (Bessel's correction).
 *   - "Replace with 1 any entry that is 0" (Algorithm 6 step 10, Algorithm 7
 *     step 24) is applied to the exact floating-point zero.
 *   - Algorithm 7 step 22's radicand can round to a small negative number;
 *     cvo_fast clamps it to 0 before the square root.
 *   - Scaling without centering divides by the standard deviation about the
 *     training mean (Section 5.1 closing remark, Table 1 first column).
 *   - The centering flags of X apply to both X^T X and X^T Y (Section 6).
 *   - Where centering is requested, Algorithms 5 and 7 form the outer product
 *     of the mean vectors first and multiply by |T| afterwards (Section 7).
 *
 * Layout: X is N x K and Y is N x M, row-major float64.  Outputs XTX are
 * P x K x K and XTY P x K x M, row-major per fold; mean and std are
 * P x (K + M), X's columns first.  std holds the factor used for scaling
 * (zeros replaced by 1); where |T| - ddof <= 0 and no scaling is requested
 * it is NaN.
 *
 * Floating point: build with -ffp-contract=off so that no multiply-add is
 * fused; every sum is accumulated left to right over rows in increasing row
 * index.  cvo_naive and cvo_naive_subset may spread their columns and output
 * rows over host threads (cvo_set_threads); each value is still formed by
 * one thread in that order, so the thread count does not change any bit.
 *
 * Parity pins: see tests/test_oracle_pins.py.  No function here is
 * "parity unpinned".
 */
#define _GNU_SOURCE 1   /* sysconf(_SC_NPROCESSORS_ONLN) */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

enum {
    CVO_OK = 0,
    CVO_INVALID_ARG = 1,
    CVO_FOLD_RANGE = 2,
    CVO_EMPTY_FOLD = 3,
    CVO_NOT_SCALABLE = 4,
    CVO_ALLOC = 5
};

enum { CVO_CENTER_X = 1, CVO_SCALE_X = 2, CVO_CENTER_Y = 4, CVO_SCALE_Y = 8 };

/* Host threads for cvo_naive / cvo_naive_subset.  Threads only split the
 * list of output columns (and of output rows of the products) between them:
 * every value is still computed by one thread with the same loop, so the
 * results are bitwise independent of the thread count. */
static int g_threads = 1;

/* Set the thread count (n <= 0: every online processor); returns the count
 * now in use. */
int cvo_set_threads(int n)
{
    if (n <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        n = c > 0 ? (int)c : 1;
    }
    g_threads = n;
    return g_threads;
}

int cvo_get_threads(void) { return g_threads; }

typedef void (*cvo_task_fn)(void *ctx, int64_t index);

struct cvo_pool_arg {
    cvo_task_fn fn;
    void *ctx;
    int64_t count, first, step;
};

static void *cvo_pool_worker(void *p)
{
    const struct cvo_pool_arg *a = (const struct cvo_pool_arg *)p;
    for (int64_t k = a->first; k < a->count; k += a->step) a->fn(a->ctx, k);
    return NULL;
}

/* fn(ctx, k) for k = 0 .. count-1, thread t taking k = t, t + T, ... (the
 * interleaving balances the triangular loops).  Falls back to the calling
 * thread alone when threads cannot be started. */
static void cvo_parallel_for(int64_t count, cvo_task_fn fn, void *ctx)
{
    int T = g_threads;
    if (T > count) T = (int)count;
    if (T <= 1) {
        for (int64_t k = 0; k < count; ++k) fn(ctx, k);
        return;
    }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)T);
    struct cvo_pool_arg *args = (struct cvo_pool_arg *)malloc(sizeof(struct cvo_pool_arg) * (size_t)T);
    int *started = (int *)calloc((size_t)T, sizeof(int));
    if (!th || !args || !started) {
        free(th); free(args); free(started);
        for (int64_t k = 0; k < count; ++k) fn(ctx, k);
        return;
    }
    for (int t = 0; t < T; ++t) {
        args[t].fn = fn; args[t].ctx = ctx; args[t].count = count; args[t].first = t; args[t].step = T;
    }
    for (int t = 1; t < T; ++t) started[t] = pthread_create(&th[t], NULL, cvo_pool_worker, &args[t]) == 0;
    cvo_pool_worker(&args[0]);
    for (int t = 1; t < T; ++t) {
        if (started[t]) pthread_join(th[t], NULL);
        else cvo_pool_worker(&args[t]);
    }
    free(th); free(args); free(started);
}

/* Algorithm 1: V[p] collects every row n with P[n] = p, visiting n in
 * increasing order.  The sets are stored as one array `rows` of length N
 * with fold p occupying rows[offsets[p] .. offsets[p+1]).  Returns
 * CVO_FOLD_RANGE for an id outside [0, P) and CVO_EMPTY_FOLD when some fold
 * has no row (Definition 1 requires the union of P[n] to be {1..P}). */
int cvo_validation_partitions(int64_t N, int32_t P, const int32_t *folds,
                              int64_t *offsets, int64_t *rows)
{
    if (N < 1 || P < 1 || !folds || !offsets || !rows) return CVO_INVALID_ARG;
    int64_t *fill = (int64_t *)calloc((size_t)P, sizeof(int64_t));
    if (!fill) return CVO_ALLOC;
    for (int32_t p = 0; p <= P; ++p) offsets[p] = 0;
    for (int64_t n = 0; n < N; ++n) {
        int32_t p = folds[n];
        if (p < 0 || p >= P) { free(fill); return CVO_FOLD_RANGE; }
        offsets[p + 1] += 1;
    }
    for (int32_t p = 0; p < P; ++p) {
        if (offsets[p + 1] == 0) { free(fill); return CVO_EMPTY_FOLD; }
        offsets[p + 1] += offsets[p];
    }
    for (int64_t n = 0; n < N; ++n) {
        int32_t p = folds[n];
        rows[offsets[p] + fill[p]] = n;
        fill[p] += 1;
    }
    free(fill);
    return CVO_OK;
}

static int check_args(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *folds,
                      const double *X, const double *Y, int flags, int ddof)
{
    if (N < 2 || K < 1 || M < 0 || P < 2 || P > N) return CVO_INVALID_ARG;
    if (!folds || !X || (M > 0 && !Y)) return CVO_INVALID_ARG;
    if (flags < 0 || flags > 15 || ddof < 0 || ddof > 1) return CVO_INVALID_ARG;
    return CVO_OK;
}

/* Column j of [X | Y] at row n (j < K: X, else Y). */
static inline double zval(const double *X, const double *Y, int32_t K, int32_t M,
                          int64_t n, int32_t j)
{
    return j < K ? X[n * (int64_t)K + j] : Y[n * (int64_t)M + (j - K)];
}

/* Training-row list T = R \ V_p in increasing row order. */
static int64_t training_rows(int64_t N, const int32_t *folds, int32_t p, int64_t *T)
{
    int64_t nt = 0;
    for (int64_t n = 0; n < N; ++n)
        if (folds[n] != p) T[nt++] = n;
    return nt;
}

/* Definition 2: column mean over the rows in T (plain left-to-right sum). */
static double column_mean(const double *X, const double *Y, int32_t K, int32_t M,
                          const int64_t *T, int64_t nt, int32_t j)
{
    double s = 0.0;
    for (int64_t t = 0; t < nt; ++t) s += zval(X, Y, K, M, T[t], j);
    return s / (double)nt;
}

/* Definition 4 with divisor |T| - ddof: two-pass sample standard deviation,
 * then Algorithm 6 step 10 (an exact zero is replaced by 1). */
static double column_std(const double *X, const double *Y, int32_t K, int32_t M,
                         const int64_t *T, int64_t nt, int32_t j, double mean, int ddof)
{
    if (nt - ddof <= 0) return NAN;
    double s = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
        double d = zval(X, Y, K, M, T[t], j) - mean;
        s += d * d;
    }
    double sd = sqrt(s / (double)(nt - ddof));
    return sd == 0.0 ? 1.0 : sd;
}

/* Preprocessed value of column j at training position t: center first
 * (Definition 3), then scale (Definition 5). */
static inline double prep(double v, double mean, double sd, int center, int scale)
{
    if (center) v = v - mean;
    if (scale) v = v / sd;
    return v;
}

static int scalable(int64_t N, int32_t P, const int32_t *folds, int flags, int ddof)
{
    if (!(flags & (CVO_SCALE_X | CVO_SCALE_Y))) return 1;
    int64_t *cnt = (int64_t *)calloc((size_t)P, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t n = 0; n < N; ++n) cnt[folds[n]] += 1;
    int ok = 1;
    for (int32_t p = 0; p < P; ++p)
        if (N - cnt[p] - ddof <= 0) ok = 0;   /* Definition 6 for ddof = 1 */
    free(cnt);
    return ok;
}

static int validate_folds(int64_t N, int32_t P, const int32_t *folds)
{
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P + 1));
    int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int rc = (off && rows) ? cvo_validation_partitions(N, P, folds, off, rows) : CVO_ALLOC;
    free(off);
    free(rows);
    return rc;
}

/* One fold of the naive algorithm, shared by the threads of its three
 * loops (columns, rows of X^T X, rows of X^T Y). */
struct naive_fold_ctx {
    const double *X, *Y;
    int32_t K, M;
    int cx, sx, cy, sy, ddof;
    const int64_t *T;
    int64_t nt;
    double *mu, *sd, *A;       /* A: preprocessed training columns, A[j * nt + t] */
    double *xtx, *xty;         /* this fold's outputs (row-major) */
};

/* Steps 7-11 for column j: training mean (Definition 2), standard deviation
 * with zero replaced by 1 (Definition 4, step 10), centering then scaling
 * (Definitions 3, 5). */
static void naive_column(void *c, int64_t jj)
{
    struct naive_fold_ctx *f = (struct naive_fold_ctx *)c;
    const int32_t j = (int32_t)jj;
    f->mu[j] = column_mean(f->X, f->Y, f->K, f->M, f->T, f->nt, j);
    f->sd[j] = column_std(f->X, f->Y, f->K, f->M, f->T, f->nt, j, f->mu[j], f->ddof);
    const int cen = j < f->K ? f->cx : f->cy, scl = j < f->K ? f->sx : f->sy;
    double *a = f->A + (int64_t)j * f->nt;
    for (int64_t t = 0; t < f->nt; ++t)
        a[t] = prep(zval(f->X, f->Y, f->K, f->M, f->T[t], j), f->mu[j], f->sd[j], cen, scl);
}

/* Step 12, row i of X^T X: dot products of column i with columns j >= i,
 * mirrored to (j, i). */
static void naive_xtx_row(void *c, int64_t ii)
{
    struct naive_fold_ctx *f = (struct naive_fold_ctx *)c;
    const int32_t i = (int32_t)ii, K = f->K;
    const double *ai = f->A + (int64_t)i * f->nt;
    for (int32_t j = i; j < K; ++j) {
        const double *aj = f->A + (int64_t)j * f->nt;
        double s = 0.0;
        for (int64_t t = 0; t < f->nt; ++t) s += ai[t] * aj[t];
        f->xtx[(int64_t)i * K + j] = s;
        f->xtx[(int64_t)j * K + i] = s;   /* a*b == b*a exactly */
    }
}

/* Step 12, row i of X^T Y. */
static void naive_xty_row(void *c, int64_t ii)
{
    struct naive_fold_ctx *f = (struct naive_fold_ctx *)c;
    const int32_t i = (int32_t)ii, K = f->K, M = f->M;
    const double *ai = f->A + (int64_t)i * f->nt;
    for (int32_t m = 0; m < M; ++m) {
        const double *bm = f->A + (int64_t)(K + m) * f->nt;
        double s = 0.0;
        for (int64_t t = 0; t < f->nt; ++t) s += ai[t] * bm[t];
        f->xty[(int64_t)i * M + m] = s;
    }
}

/* Algorithms 2 / 4 / 6 for the folds listed in `sel` (all P folds when sel
 * is NULL).  For each fold p: T = R \ V_p (step 5), X_T and Y_T (step 6),
 * training means (step 7), centering (step 8), training standard deviations
 * with zeros replaced by 1 (steps 9-10), scaling (step 11), products
 * (step 12).  Outputs of folds not listed are left untouched. */
static int naive_folds(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *folds,
                       const double *X, const double *Y, int flags, int ddof,
                       const int32_t *sel, int32_t nsel,
                       double *XTX, double *XTY, double *mean_out, double *std_out)
{
    int rc = check_args(N, K, M, P, folds, X, Y, flags, ddof);
    if (rc) return rc;
    if ((rc = validate_folds(N, P, folds))) return rc;
    int sc = scalable(N, P, folds, flags, ddof);
    if (sc < 0) return CVO_ALLOC;
    if (!sc) return CVO_NOT_SCALABLE;
    const int32_t count = sel ? nsel : P;
    for (int32_t q = 0; q < count; ++q)
        if (sel && (sel[q] < 0 || sel[q] >= P)) return CVO_INVALID_ARG;

    const int32_t D = K + M;
    struct naive_fold_ctx f;
    f.X = X; f.Y = Y; f.K = K; f.M = M; f.ddof = ddof;
    f.cx = !!(flags & CVO_CENTER_X); f.sx = !!(flags & CVO_SCALE_X);
    f.cy = !!(flags & CVO_CENTER_Y); f.sy = !!(flags & CVO_SCALE_Y);
    int64_t *T = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    double *mu = (double *)malloc(sizeof(double) * (size_t)D);
    double *sd = (double *)malloc(sizeof(double) * (size_t)D);
    double *A = (double *)malloc(sizeof(double) * (size_t)D * (size_t)N);
    if (!T || !mu || !sd || !A) { free(T); free(mu); free(sd); free(A); return CVO_ALLOC; }
    f.T = T; f.mu = mu; f.sd = sd; f.A = A;

    for (int32_t q = 0; q < count; ++q) {
        const int32_t p = sel ? sel[q] : q;
        f.nt = training_rows(N, folds, p, T);
        cvo_parallel_for(D, naive_column, &f);
        if (mean_out) for (int32_t j = 0; j < D; ++j) mean_out[(int64_t)p * D + j] = mu[j];
        if (std_out) for (int32_t j = 0; j < D; ++j) std_out[(int64_t)p * D + j] = sd[j];
        if (XTX) {
            f.xtx = XTX + (int64_t)p * K * K;
            cvo_parallel_for(K, naive_xtx_row, &f);
        }
        if (XTY && M > 0) {
            f.xty = XTY + (int64_t)p * K * M;
            cvo_parallel_for(K, naive_xty_row, &f);
        }
    }
    free(T); free(mu); free(sd); free(A);
    return CVO_OK;
}

/* Algorithms 2 / 4 / 6 generalised to every flag combination, all folds. */
int cvo_naive(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *folds,
              const double *X, const double *Y, int flags, int ddof,
              double *XTX, double *XTY, double *mean_out, double *std_out)
{
    return naive_folds(N, K, M, P, folds, X, Y, flags, ddof, NULL, 0, XTX, XTY, mean_out, std_out);
}

/* The same for the nsel folds listed in sel (outputs are still P-sized). */
int cvo_naive_subset(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *folds,
                     const double *X, const double *Y, int flags, int ddof,
                     const int32_t *sel, int32_t nsel,
                     double *XTX, double *XTY, double *mean_out, double *std_out)
{
    if (!sel || nsel < 1) return CVO_INVALID_ARG;
    return naive_folds(N, K, M, P, folds, X, Y, flags, ddof, sel, nsel, XTX, XTY, mean_out, std_out);
}

/* One entry of cvo_naive's output for fold p: which = 0 selects
 * XTX[p][i][j] (0 <= i, j < K), which = 1 selects XTY[p][i][j]
 * (0 <= i < K, 0 <= j < M).  Same arithmetic and order as cvo_naive; the
 * result is written to *out.  Does not re-validate the whole partitioning
 * beyond the fold being non-empty and scalable. */
int cvo_naive_entry(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *folds,
                    const double *X, const double *Y, int flags, int ddof,
                    int32_t p, int which, int32_t i, int32_t j, double *out)
{
    int rc = check_args(N, K, M, P, folds, X, Y, flags, ddof);
    if (rc) return rc;
    if (p < 0 || p >= P || i < 0 || i >= K || !out) return CVO_INVALID_ARG;
    if (which == 0 ? (j < 0 || j >= K) : (which != 1 || j < 0 || j >= M)) return CVO_INVALID_ARG;
    int64_t *T = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!T) return CVO_ALLOC;
    const int64_t nt = training_rows(N, folds, p, T);
    if (nt == N) { free(T); return CVO_EMPTY_FOLD; }
    if ((flags & (CVO_SCALE_X | CVO_SCALE_Y)) && nt - ddof <= 0) { free(T); return CVO_NOT_SCALABLE; }
    const int cx = !!(flags & CVO_CENTER_X), sx = !!(flags & CVO_SCALE_X);
    const int cy = !!(flags & CVO_CENTER_Y), sy = !!(flags & CVO_SCALE_Y);
    const int32_t jj = which == 0 ? j : K + j;
    const double mi = column_mean(X, Y, K, M, T, nt, i);
    const double si = column_std(X, Y, K, M, T, nt, i, mi, ddof);
    const double mj = column_mean(X, Y, K, M, T, nt, jj);
    const double sj = column_std(X, Y, K, M, T, nt, jj, mj, ddof);
    const int cj = which == 0 ? cx : cy, sjf = which == 0 ? sx : sy;
    double s = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
        const double a = prep(zval(X, Y, K, M, T[t], i), mi, si, cx, sx);
        const double b = prep(zval(X, Y, K, M, T[t], jj), mj, sj, cj, sjf);
        s += a * b;
    }
    *out = s;
    free(T);
    return CVO_OK;
}

/* Algorithms 3 / 5 / 7 generalised to every flag combination (Table 1). */
int cvo_fast(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *folds,
             const double *X, const double *Y, int flags, int ddof,
             double *XTX, double *XTY, double *mean_out, double *std_out)
{
    int rc = check_args(N, K, M, P, folds, X, Y, flags, ddof);
    if (rc) return rc;
    int sc = 1;

    const int cx = !!(flags & CVO_CENTER_X), sx = !!(flags & CVO_SCALE_X);
    const int cy = !!(flags & CVO_CENTER_Y), sy = !!(flags & CVO_SCALE_Y);
    const int64_t KK = (int64_t)K * K, KM = (int64_t)K * M;

    /* Step 2: Algorithm 1. */
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P + 1));
    int64_t *V = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    double *xtx = (double *)calloc((size_t)KK, sizeof(double));
    double *xty = (double *)calloc((size_t)(KM > 0 ? KM : 1), sizeof(double));
    double *xtxv = (double *)malloc(sizeof(double) * (size_t)KK);
    double *xtyv = (double *)malloc(sizeof(double) * (size_t)(KM > 0 ? KM : 1));
    double *vec = (double *)calloc((size_t)(K + M) * 12, sizeof(double));
    if (!off || !V || !xtx || !xty || !xtxv || !xtyv || !vec) { rc = CVO_ALLOC; goto done; }
    if ((rc = cvo_validation_partitions(N, P, folds, off, V))) goto done;
    sc = scalable(N, P, folds, flags, ddof);
    if (sc < 0) { rc = CVO_ALLOC; goto done; }
    if (!sc) { rc = CVO_NOT_SCALABLE; goto done; }
    {
        double *mux = vec, *muy = mux + K;                 /* step 3 means */
        double *sumx = muy + M, *sumy = sumx + K;          /* step 4 */
        double *sqx = sumy + M, *sqy = sqx + K;
        double *muxv = sqy + M, *muyv = muxv + K;          /* step 10 */
        double *muxt = muyv + M, *muyt = muxt + K;         /* steps 12-13 */
        double *sdxt = muyt + M, *sdyt = sdxt + K;         /* steps 22-24 */
        double *sumxv = sdyt + M, *sumyv = sumxv + K;      /* step 17 */
        double *sqxv = sumyv + M, *sqyv = sqxv + K;        /* step 19 */

        /* Step 3: XTX = X^T X, XTY = X^T Y over every row; mean rows. */
        for (int64_t n = 0; n < N; ++n) {
            const double *x = X + n * K;
            const double *y = M > 0 ? Y + n * M : NULL;
            for (int32_t i = 0; i < K; ++i) {
                for (int32_t j = i; j < K; ++j) xtx[(int64_t)i * K + j] += x[i] * x[j];
                for (int32_t m = 0; m < M; ++m) xty[(int64_t)i * M + m] += x[i] * y[m];
            }
        }
        for (int32_t i = 0; i < K; ++i)
            for (int32_t j = 0; j < i; ++j) xtx[(int64_t)i * K + j] = xtx[(int64_t)j * K + i];
        /* Step 4: column sums and sums of squares over every row. */
        for (int64_t n = 0; n < N; ++n) {
            for (int32_t i = 0; i < K; ++i) { double v = X[n * K + i]; sumx[i] += v; sqx[i] += v * v; }
            for (int32_t m = 0; m < M; ++m) { double v = Y[n * M + m]; sumy[m] += v; sqy[m] += v * v; }
        }
        for (int32_t i = 0; i < K; ++i) mux[i] = sumx[i] / (double)N;
        for (int32_t m = 0; m < M; ++m) muy[m] = sumy[m] / (double)N;

        for (int32_t p = 0; p < P; ++p) {
            const int64_t *v = V + off[p];
            const int64_t nv = off[p + 1] - off[p];       /* step 11 */
            const int64_t nt = N - nv;
            /* Steps 7-8: products over the validation rows only. */
            memset(xtxv, 0, sizeof(double) * (size_t)KK);
            if (KM > 0) memset(xtyv, 0, sizeof(double) * (size_t)KM);
            for (int64_t r = 0; r < nv; ++r) {
                const double *x = X + v[r] * K;
                const double *y = M > 0 ? Y + v[r] * M : NULL;
                for (int32_t i = 0; i < K; ++i) {
                    for (int32_t j = i; j < K; ++j) xtxv[(int64_t)i * K + j] += x[i] * x[j];
                    for (int32_t m = 0; m < M; ++m) xtyv[(int64_t)i * M + m] += x[i] * y[m];
                }
            }
            for (int32_t i = 0; i < K; ++i)
                for (int32_t j = 0; j < i; ++j) xtxv[(int64_t)i * K + j] = xtxv[(int64_t)j * K + i];
            /* Step 10: validation means; steps 17 and 19: validation sums. */
            for (int32_t i = 0; i < K; ++i) { sumxv[i] = 0.0; sqxv[i] = 0.0; }
            for (int32_t m = 0; m < M; ++m) { sumyv[m] = 0.0; sqyv[m] = 0.0; }
            for (int64_t r = 0; r < nv; ++r) {
                for (int32_t i = 0; i < K; ++i) { double a = X[v[r] * K + i]; sumxv[i] += a; sqxv[i] += a * a; }
                for (int32_t m = 0; m < M; ++m) { double a = Y[v[r] * M + m]; sumyv[m] += a; sqyv[m] += a * a; }
            }
            for (int32_t i = 0; i < K; ++i) muxv[i] = sumxv[i] / (double)nv;
            for (int32_t m = 0; m < M; ++m) muyv[m] = sumyv[m] / (double)nv;
            /* Steps 12-13 (Lemmas 7, 8): training means by downdating. */
            const double a = (double)N / (double)nt, b = (double)nv / (double)nt;
            for (int32_t i = 0; i < K; ++i) muxt[i] = a * mux[i] - b * muxv[i];
            for (int32_t m = 0; m < M; ++m) muyt[m] = a * muy[m] - b * muyv[m];
            /* Steps 18, 20-24 (Lemmas 12-14): training standard deviations. */
            for (int32_t i = 0; i < K; ++i) {
                const double st = sumx[i] - sumxv[i], qt = sqx[i] - sqxv[i];
                double num = (double)nt * (muxt[i] * muxt[i]) + qt - 2.0 * muxt[i] * st;
                if (num < 0.0) num = 0.0;
                double sd = nt - ddof > 0 ? sqrt(num / (double)(nt - ddof)) : NAN;
                sdxt[i] = sd == 0.0 ? 1.0 : sd;
            }
            for (int32_t m = 0; m < M; ++m) {
                const double st = sumy[m] - sumyv[m], qt = sqy[m] - sqyv[m];
                double num = (double)nt * (muyt[m] * muyt[m]) + qt - 2.0 * muyt[m] * st;
                if (num < 0.0) num = 0.0;
                double sd = nt - ddof > 0 ? sqrt(num / (double)(nt - ddof)) : NAN;
                sdyt[m] = sd == 0.0 ? 1.0 : sd;
            }
            if (mean_out) {
                for (int32_t i = 0; i < K; ++i) mean_out[(int64_t)p * (K + M) + i] = muxt[i];
                for (int32_t m = 0; m < M; ++m) mean_out[(int64_t)p * (K + M) + K + m] = muyt[m];
            }
            if (std_out) {
                for (int32_t i = 0; i < K; ++i) std_out[(int64_t)p * (K + M) + i] = sdxt[i];
                for (int32_t m = 0; m < M; ++m) std_out[(int64_t)p * (K + M) + K + m] = sdyt[m];
            }
            /* Step 9: subtract; steps 14-16: rank-one centering (outer
             * product first, then times |T|); steps 25-27: Hadamard division. */
            if (XTX) {
                double *out = XTX + (int64_t)p * KK;
                for (int32_t i = 0; i < K; ++i)
                    for (int32_t j = 0; j < K; ++j) {
                        double g = xtx[(int64_t)i * K + j] - xtxv[(int64_t)i * K + j];
                        if (cx) g = g - (double)nt * (muxt[i] * muxt[j]);
                        if (sx) g = g / (sdxt[i] * sdxt[j]);
                        out[(int64_t)i * K + j] = g;
                    }
            }
            if (XTY && M > 0) {
                double *out = XTY + (int64_t)p * KM;
                for (int32_t i = 0; i < K; ++i)
                    for (int32_t m = 0; m < M; ++m) {
                        double g = xty[(int64_t)i * M + m] - xtyv[(int64_t)i * M + m];
                        if (cx || cy) g = g - (double)nt * (muxt[i] * muyt[m]);
                        const double di = sx ? sdxt[i] : 1.0, dm = sy ? sdyt[m] : 1.0;
                        if (sx || sy) g = g / (di * dm);
                        out[(int64_t)i * M + m] = g;
                    }
            }
        }
    }
    rc = CVO_OK;
done:
    free(off); free(V); free(xtx); free(xty); free(xtxv); free(xtyv); free(vec);
    return rc;
}

/* ------------------------------------------------------------------------
 * Models on the products: per-fold ridge regression / ordinary least squares
 * through the normal equations, and its error on the validation partition.
 * The paper names RR and OLS via the normal equations as consumers of
 * X^T X and X^T Y (Section 1) and cross-validation as fitting on each
 * training partition and evaluating on its validation partition (Section 1).
 *
 * Readings (the paper does not fix them):
 *   - The model lives in the space the products were preprocessed into: for
 *     fold p, B_p = (XTX_p + lambda I)^-1 XTY_p with XTX_p, XTY_p as returned
 *     for the flags (lambda = 0 is OLS).
 *   - A validation row is preprocessed with the same fold's TRAINING
 *     statistics (no leakage): x~_k = (x_k - [cX] mean_k) / ([sX] ? std_k : 1),
 *     likewise y~.  The prediction y~^ = x~ B_p is mapped back to Y's units:
 *     y^ = y~^ ([sY] ? std : 1) + ([cY] ? mean : 0).  Without cY nothing is
 *     added back, which is what a model fitted on uncentered Y predicts.
 *   - press[p][m] = sum over the validation rows n of fold p of
 *     (y_nm - y^_nm)^2, rows in increasing index order.
 */

/* For each fold p: the Cholesky factorisation XTX_p + lambda I = L L^T,
 * column by column (L[j][j] = sqrt(a_jj + lambda - sum_{k<j} L[j][k]^2),
 * L[i][j] = (a_ij - sum_{k<j} L[i][k] L[j][k]) / L[j][j] for i > j, sums in
 * increasing k), then L z = c by forward and L^T b = z by back substitution
 * for each of the M columns of XTY_p.  Only the lower triangle of XTX_p is
 * read.  info[p] = 0, or j + 1 when the pivot of column j is not positive
 * (then B_p is set to NaN).  B is P x K x M row-major. */
int cvo_ridge(int32_t P, int32_t K, int32_t M, const double *XTX, const double *XTY, double lambda,
              double *B, int32_t *info) {
    if (P < 1 || K < 1 || M < 0 || !XTX || !B || !info || (M > 0 && !XTY)) return CVO_INVALID_ARG;
    double *L = (double *)malloc(sizeof(double) * (size_t)K * (size_t)K);
    double *z = (double *)malloc(sizeof(double) * (size_t)K);
    if (!L || !z) {
        free(L);
        free(z);
        return CVO_ALLOC;
    }
    for (int32_t p = 0; p < P; ++p) {
        const double *A = XTX + (int64_t)p * K * K;
        const double *C = XTY ? XTY + (int64_t)p * K * M : NULL;
        double *Bp = B + (int64_t)p * K * M;
        info[p] = 0;
        for (int32_t j = 0; j < K && info[p] == 0; ++j) {
            double s = A[(int64_t)j * K + j] + lambda;
            for (int32_t k = 0; k < j; ++k) s -= L[(int64_t)j * K + k] * L[(int64_t)j * K + k];
            if (!(s > 0.0)) {
                info[p] = j + 1;
                break;
            }
            const double d = sqrt(s);
            L[(int64_t)j * K + j] = d;
            for (int32_t i = j + 1; i < K; ++i) {
                double t = A[(int64_t)i * K + j];
                for (int32_t k = 0; k < j; ++k) t -= L[(int64_t)i * K + k] * L[(int64_t)j * K + k];
                L[(int64_t)i * K + j] = t / d;
            }
        }
        if (info[p] != 0) {
            for (int64_t e = 0; e < (int64_t)K * M; ++e) Bp[e] = NAN;
            continue;
        }
        for (int32_t m = 0; m < M; ++m) {
            for (int32_t i = 0; i < K; ++i) {
                double t = C[(int64_t)i * M + m];
                for (int32_t k = 0; k < i; ++k) t -= L[(int64_t)i * K + k] * z[k];
                z[i] = t / L[(int64_t)i * K + i];
            }
            for (int32_t i = K - 1; i >= 0; --i) {
                double t = z[i];
                for (int32_t k = i + 1; k < K; ++k) t -= L[(int64_t)k * K + i] * Bp[(int64_t)k * M + m];
                Bp[(int64_t)i * M + m] = t / L[(int64_t)i * K + i];
            }
        }
    }
    free(L);
    free(z);
    return CVO_OK;
}

/* Validation error of the per-fold models (readings above).  mean and std are
 * P x (K + M) as returned with the products (X's columns first), B is
 * P x K x M, press is P x M. */
int cvo_press(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *folds, const double *X,
              const double *Y, int flags, const double *mean, const double *std, const double *B,
              double *press) {
    if (N < 1 || K < 1 || M < 1 || P < 1 || !folds || !X || !Y || !mean || !std || !B || !press)
        return CVO_INVALID_ARG;
    const int cx = (flags & CVO_CENTER_X) != 0, sx = (flags & CVO_SCALE_X) != 0;
    const int cy = (flags & CVO_CENTER_Y) != 0, sy = (flags & CVO_SCALE_Y) != 0;
    const int32_t KM = K + M;
    for (int64_t e = 0; e < (int64_t)P * M; ++e) press[e] = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        const int32_t p = folds[n];
        if (p < 0 || p >= P) return CVO_FOLD_RANGE;
        const double *mu = mean + (int64_t)p * KM, *sd = std + (int64_t)p * KM;
        const double *Bp = B + (int64_t)p * K * M;
        for (int32_t m = 0; m < M; ++m) {
            double pred = 0.0;
            for (int32_t k = 0; k < K; ++k) {
                double xt = X[n * K + k];
                if (cx) xt -= mu[k];
                if (sx) xt /= sd[k];
                pred += xt * Bp[(int64_t)k * M + m];
            }
            double yhat = pred;
            if (sy) yhat *= sd[K + m];
            if (cy) yhat += mu[K + m];
            const double r = Y[n * M + m] - yhat;
            press[(int64_t)p * M + m] += r * r;
        }
    }
    return CVO_OK;
}
