/*
 * cvx.h -- C ABI of the GB300 library for fast partition-based
 * cross-validation products with training-partition centering and scaling.
 *
 * The method is Engstrom & Jensen, "Fast Partition-Based Cross-Validation
 * With Centering and Scaling for X^T X and X^T Y" (arXiv 2401.13185).
 *
 * Problem statement (Section 3, Definition 1): X is N x K, Y is N x M, and a
 * partitioning assigns every row n to one of P folds.  For every fold p the
 * training partition T_p is every row not in fold p.  The library returns,
 * for every p, the products X_T^T X_T (K x K) and X_T^T Y_T (K x M) where
 * X_T and Y_T are optionally centered by their training-partition column
 * means (Definitions 2, 3) and optionally scaled by their training-partition
 * column standard deviations (Definitions 4, 5), in any of the 16
 * combinations of Section 6 / Table 1.  Statistics come from the training
 * rows only, so no validation row leaks into its own fold's preprocessing.
 * On top of the products, cv_ridge / cv_ridge_press fit the per-fold ridge
 * or OLS models the paper names as consumers (Section 1) and measure their
 * error on each validation partition.
 *
 * Threading: calls on different plans may run concurrently from different
 * host threads.  A single plan must not be used by two calls at once.
 *
 * Errors: every function returns a cv_status and never throws.  A CUDA
 * runtime error inside a call is returned as CV_ERR_CUDA.
 */
#ifndef CVX_H
#define CVX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CV_OK = 0,
    CV_ERR_INVALID_ARG = 1,   /* bad scalar, null pointer, bad layout or alignment */
    CV_ERR_FOLD_RANGE = 2,    /* a fold id outside [0, P) (Definition 1) */
    CV_ERR_EMPTY_FOLD = 3,    /* a fold with no row (Definition 1) */
    CV_ERR_NOT_SCALABLE = 4,  /* scaling requested and some |T_p| - ddof < 1 (Definition 6) */
    CV_ERR_ALLOC = 5,         /* device or host allocation failed */
    CV_ERR_CUDA = 6,          /* a CUDA runtime call failed */
    CV_ERR_UNSUPPORTED = 7,   /* valid request this build does not implement */
    CV_ERR_TIMEOUT = 8,       /* a bounded device-side wait expired */
    CV_ERR_RANGE = 9          /* split-precision operand out of the FP16 range */
} cv_status;

/* Preprocessing flags (Section 6).  Centering subtracts the training column
 * mean, scaling divides by the training column standard deviation; when both
 * are set, centering comes first.  X's flags apply to X^T X and X^T Y alike. */
enum { CV_CENTER_X = 1, CV_SCALE_X = 2, CV_CENTER_Y = 4, CV_SCALE_Y = 8 };

typedef enum { CV_F32 = 0, CV_F64 = 1 } cv_dtype;

/* Arithmetic of the Gram contraction.  Every tensor-core precision works on
 * the shifted, power-of-two scaled values v = (x - s) 2^e of each column (s a
 * sampled column mean), keeps the column sums and sums of squares in the same
 * contraction, and computes the statistics in FP64.
 *   CV_PREC_FP64    FP64 fused multiply-add on the CUDA cores; statistics and
 *                   epilogue in FP64 (relative error ~1e-15).
 *   CV_PREC_FP16X3  tcgen05 tensor cores: v is split into an integer part
 *                   hi = rint(v) and a remainder lo, both FP16 (about 22
 *                   significant bits in all).  hi*hi accumulates exactly in
 *                   its own FP32 tensor memory accumulator, the three
 *                   correction products hi*lo + lo*hi + lo*lo in a second;
 *                   fold sums are exact int64 plus FP32, the centering /
 *                   scaling epilogue FP32 (relative error ~1e-7 on the
 *                   products).
 *   CV_PREC_BF16X3  tcgen05 tensor cores: hi = bf16(v), lo = bf16(v - hi);
 *                   hi*hi + hi*lo + lo*hi in one FP32 accumulator (three
 *                   products, lo*lo dropped: about 2^-16 relative).
 *   CV_PREC_TF32    tcgen05 tensor cores: one product of tf32(v) (10-bit
 *                   mantissa) in an FP32 accumulator; the fastest, about
 *                   1e-4 relative.
 *   CV_PREC_TF32X3  tcgen05 tensor cores: hi = tf32(v), lo = tf32(v - hi)
 *                   (about 22 significant bits); hi*hi + hi*lo + lo*hi in
 *                   FP32 accumulators (three TF32 products, lo*lo dropped:
 *                   about 2^-22 relative), each at half the FP16 rate.
 *   CV_PREC_AUTO    CV_PREC_FP16X3. */
typedef enum {
    CV_PREC_FP64 = 0,
    CV_PREC_TF32 = 1,
    CV_PREC_TF32X3 = 2,
    CV_PREC_BF16X3 = 3,
    CV_PREC_FP16X3 = 4,
    CV_PREC_AUTO = 5
} cv_precision;

typedef struct cv_plan_s *cv_plan_t;

/*
 * cv_plan -- Algorithm 1 (Section 3): bucket the rows by fold.
 *
 *   out           receives the plan handle (owned by the caller, released with
 *                 cv_plan_destroy).
 *   N, K, M, P    rows, X columns, Y columns (M may be 0), folds;
 *                 2 <= P <= N, K >= 1, N < 2^31.
 *   fold_ids      int32[N], fold of each row, values in [0, P) (the paper's
 *                 partition p is fold p - 1).  Device pointer when
 *                 fold_ids_on_device != 0, host pointer otherwise.  Read
 *                 during the call only; the plan keeps its own copy of what
 *                 it needs.
 *   in_dtype      element type of X and Y passed to cv_products.
 *   out_dtype     element type of the XTX / XTY outputs.
 *   prec          Gram arithmetic (cv_precision).
 *   stream        cudaStream_t for the plan's device work (NULL = legacy
 *                 default stream).
 *
 * On the device the plan runs a fold histogram (validating every id) and a
 * stable counting sort that lists the rows of each fold in increasing row
 * order.  It synchronises `stream` once to read the P fold sizes back, and
 * allocates all device workspace that cv_products needs, so cv_products
 * itself never allocates.
 *
 * Strategy: when the folds average more than 64 rows, every fold's part of
 * the Gram is reduced from per-segment tiles (Algorithm 7 as written).  With
 * smaller folds (many folds, up to leave-one-out) only the Gram over all rows
 * is reduced and each fold's part is recomputed from its rows inside the
 * epilogue, so the workspace holds no per-fold tiles.
 *
 * Errors: CV_ERR_INVALID_ARG (scalars, null pointers), CV_ERR_FOLD_RANGE,
 * CV_ERR_EMPTY_FOLD, CV_ERR_UNSUPPORTED (a workspace larger than this build
 * supports), CV_ERR_ALLOC, CV_ERR_CUDA.  On error *out
 * is set to NULL and nothing is leaked.
 */
cv_status cv_plan(cv_plan_t *out, int64_t N, int32_t K, int32_t M, int32_t P,
                  const int32_t *fold_ids, int fold_ids_on_device,
                  cv_dtype in_dtype, cv_dtype out_dtype, cv_precision prec,
                  void *stream);

/*
 * Plan options (cv_plan_ex).  A zero-initialised struct gives the defaults.
 * strategy and ctas do not change what is computed, only how the work is cut
 * up, and with it the rounding of the split precisions' FP32 partial sums:
 * two plans with equal shapes, fold ids, precision and options give bitwise
 * equal results on devices with the same SM count (with ctas set explicitly,
 * on any device of this architecture).
 *
 *   strategy      CV_STRATEGY_AUTO: the rule described under cv_plan;
 *                 CV_STRATEGY_FOLD_GROUPED: per-fold tiles (Algorithm 7 as
 *                 written) whatever the fold sizes;
 *                 CV_STRATEGY_SMALL_FOLDS: the small-fold strategy (only H
 *                 over all rows is reduced, each fold's part is recomputed
 *                 from its rows in the epilogue) whatever the fold sizes; not
 *                 with a fold range.
 *   ctas          the number of concurrently running contraction CTAs the
 *                 segment lengths are tuned for (longer segments when fewer:
 *                 fewer partial tiles to write and reduce).  0: every SM of
 *                 the device.  A caller that runs several plans side by side
 *                 gives each its share.
 *   fold_begin, fold_end
 *                 0, 0: the plan computes every fold.  Otherwise the plan
 *                 owns folds [fold_begin, fold_end) of the P folds (one shard
 *                 of a fold-sharded computation over several GPUs, Lemma 2:
 *                 the Gram over all rows is the sum of the folds' Grams).
 *                 Such a plan reads only its folds' rows (and the shift
 *                 estimate's fixed row sample), is run with
 *                 cv_products_partial and cv_finalize_total (not
 *                 cv_products), writes outputs for its folds only (fold
 *                 fold_begin + q at index q), and always takes the
 *                 fold-grouped strategy.  Every shard of one computation must
 *                 use the same N, K, M, P, fold ids, dtypes, precision and
 *                 ctas, so that all of them cut segments and scale operands
 *                 alike and their partial totals add up.
 *   xtx_layout    CV_XTX_FULL: each fold's X^T X as K x K row-major, both
 *                 triangles.  CV_XTX_PACKED_UPPER: only its upper triangle,
 *                 row by row (entry (i, j), i <= j, at
 *                 i K - i (i - 1) / 2 + (j - i)), K (K + 1) / 2 values per
 *                 fold: half the bytes where the outputs dominate.
 *   wait_limit_ns the bound of every wait inside the tensor-core kernels
 *                 (an operand copy, an MMA, a drained accumulator), after
 *                 which the kernel stops, frees its tensor memory and records
 *                 CV_ERR_TIMEOUT for cv_plan_status.  0: one second.
 */
#define CV_STRATEGY_AUTO 0
#define CV_STRATEGY_FOLD_GROUPED 1
#define CV_STRATEGY_SMALL_FOLDS 2
#define CV_XTX_FULL 0
#define CV_XTX_PACKED_UPPER 1

typedef struct cv_plan_options {
    int32_t strategy;
    int32_t ctas;
    int32_t fold_begin, fold_end;
    int32_t xtx_layout;
    int32_t reserved;      /* must be 0 */
    int64_t wait_limit_ns;
} cv_plan_options;

/*
 * cv_plan_ex -- cv_plan with options; opts == NULL is cv_plan.  Errors as
 * cv_plan, and CV_ERR_INVALID_ARG for an unknown strategy or layout, ctas < 0,
 * wait_limit_ns < 0, reserved != 0, or a fold range that is not empty (0, 0)
 * and not 0 <= fold_begin < fold_end <= P (or set with
 * CV_STRATEGY_SMALL_FOLDS).
 */
cv_status cv_plan_ex(cv_plan_t *out, int64_t N, int32_t K, int32_t M, int32_t P,
                     const int32_t *fold_ids, int fold_ids_on_device,
                     cv_dtype in_dtype, cv_dtype out_dtype, cv_precision prec,
                     const cv_plan_options *opts, void *stream);

/*
 * Tuning: which plan options (strategy, ctas) run a problem fastest on this
 * device, measured, and remembered in a JSON cache file.
 *
 * cv_tune_key -- the cache key of a problem shape: the device's SM count,
 * the precision, the dtypes, K, M, and N and the mean fold size N / P each
 * rounded down to a power of two, e.g.
 * "sm152/prec4/in0/out1/K1024/M16/N2^19/rows2^15".  Writes at most `size`
 * bytes including the terminating zero.  Errors: CV_ERR_INVALID_ARG (null
 * pointer, size too small, a scalar out of range), CV_ERR_CUDA (no device).
 *
 * cv_tune_cache_get / cv_tune_cache_put -- look up or record the options
 * and time (ms per cv_products call) for `key` in the JSON cache at `path`
 * (NULL: the file named by the environment variable CVX_TUNE_CACHE; with
 * neither, get reports CV_ERR_UNSUPPORTED and put does nothing).  The file
 * is one JSON object mapping keys to {"strategy": s, "ctas": c, "ms": t};
 * put rewrites it with the entry added or replaced (entries it cannot parse
 * are dropped; the new file replaces the old one by a rename).  Keys use
 * the characters [A-Za-z0-9/^_.-] only.  Errors: CV_ERR_INVALID_ARG (a bad
 * key, options or time; for put also a file that cannot be written);
 * get: CV_ERR_UNSUPPORTED when the key is absent or the file is missing or
 * unreadable.  Host only: neither touches the device.
 *
 * cv_plan_tune -- time cv_products for the candidate options of this
 * problem and return the fastest in *best (fold range, layout and wait limit
 * zero) and its time in *best_ms (may be NULL).  Candidates: the default
 * (CV_STRATEGY_AUTO, every SM), the fold-grouped strategy with half of the
 * SMs' worth of segments, and, for folds averaging at most 256 rows, both
 * explicit strategies.  With a cache (path or CVX_TUNE_CACHE) a cached entry
 * for the problem's key is returned without measuring, and a measured
 * result is recorded.  Arguments as cv_plan and cv_products (outputs are
 * workspace the tuner allocates and frees; the inputs stay unchanged).
 * Synchronises `stream`; not capturable.  Errors: those of cv_plan_ex and
 * cv_products, CV_ERR_ALLOC.
 */
cv_status cv_tune_key(int64_t N, int32_t K, int32_t M, int32_t P, cv_dtype in_dtype, cv_dtype out_dtype,
                      cv_precision prec, char *key, int32_t size);
cv_status cv_tune_cache_get(const char *path, const char *key, cv_plan_options *opts, double *ms);
cv_status cv_tune_cache_put(const char *path, const char *key, const cv_plan_options *opts, double ms);
cv_status cv_plan_tune(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *fold_ids,
                       int fold_ids_on_device, cv_dtype in_dtype, cv_dtype out_dtype, cv_precision prec,
                       const void *X, int64_t ldx, const void *Y, int64_t ldy, int flags, int ddof,
                       const char *cache_path, cv_plan_options *best, double *best_ms, void *stream);

/*
 * cv_products -- Algorithm 7 (Section 5) generalised to all 16 flag
 * combinations (Section 6, Table 1): for every fold p,
 *
 *   XTX[p] = A_p^T A_p,  XTY[p] = A_p^T B_p,
 *
 * where A_p / B_p are X_T / Y_T centered (if CV_CENTER_X / CV_CENTER_Y) and
 * then divided by their column standard deviations (if CV_SCALE_X /
 * CV_SCALE_Y), all statistics over T_p.  The standard deviation divides by
 * |T_p| - ddof; a zero standard deviation is replaced by 1 (Algorithm 7
 * step 24).  Centering X or Y alone already centers X^T Y (Lemma 9).
 *
 *   plan          from cv_plan.
 *   X, ldx        device pointer to X, row-major N x K with leading
 *                 dimension ldx >= K elements, of the plan's in_dtype.
 *   Y, ldy        device pointer to Y (N x M, ldy >= M); may be NULL when
 *                 M == 0.
 *   flags         bitwise OR of CV_CENTER_X, CV_SCALE_X, CV_CENTER_Y,
 *                 CV_SCALE_Y (0..15).
 *   ddof          0 or 1 (1 = Bessel's correction, Definition 4).
 *   XTX           device pointer, P x K x K row-major (fold-major), of the
 *                 plan's out_dtype, or NULL to skip.  Both triangles are
 *                 written and are bitwise symmetric.  With the plan option
 *                 CV_XTX_PACKED_UPPER: P x K (K + 1) / 2, each fold's upper
 *                 triangle row by row.
 *   XTY           device pointer, P x K x M row-major, or NULL to skip.
 *   mean_out      optional device pointer, P x (K + M) doubles: training
 *                 column means of X then Y.
 *   std_out       optional device pointer, P x (K + M) doubles: training
 *                 column standard deviations as used for scaling (zeros
 *                 replaced by 1).
 *   stream        cudaStream_t (NULL = legacy default stream).
 *
 * All work is enqueued on `stream`; the call does not synchronise and does
 * not allocate.  Outputs are complete when the stream reaches that point.
 * The call can be captured into a CUDA graph on `stream` (unless the plan is
 * profiling); replays read the captured input and output addresses.
 * Buffers are owned by the caller and must stay valid until then.
 * The plan's workspace holds the call's intermediate results (and, for
 * cv_finalize, its fold sums), so calls on one plan must not overlap on the
 * device: issue them on one stream, or order them with events.
 *
 * Errors (returned synchronously): CV_ERR_INVALID_ARG (null plan, a
 * sharded plan, bad flags / ddof / ld, null X, Y missing with M > 0, output
 * buffer overlap is not checked), CV_ERR_NOT_SCALABLE (a scale flag is set and some fold
 * has |T_p| - ddof < 1, Definition 6), CV_ERR_CUDA (launch failure).
 * Errors found on the device (CV_ERR_RANGE: a split-precision operand after
 * shifting exceeded the FP16 range, outputs are then invalid) are recorded
 * in the plan and returned by cv_plan_status.
 */
cv_status cv_products(cv_plan_t plan, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                      int flags, int ddof, void *XTX, void *XTY,
                      double *mean_out, double *std_out, void *stream);

/*
 * cv_finalize -- the products and statistics of cv_products for other
 * flags or ddof, from the fold sums the plan's last cv_products left behind:
 * only the statistics (Algorithm 7 steps 11-13, 18, 20-24) and the epilogue
 * (steps 9, 14-16, 25-27) run again.  All 16 combinations of Section 6 /
 * Table 1 differ only in these cheap corrections (Propositions 15, 16), so a
 * sweep over them costs one contraction and 16 bandwidth-bound epilogues.
 *
 *   plan          a plan on which cv_products has been called; the call's
 *                 work must precede this one on the stream (or be complete).
 *   X, ldx, Y, ldy  the inputs of that cv_products call.  Read only by plans
 *                 that take the small-fold strategy (folds averaging at most
 *                 64 rows, or CV_STRATEGY_SMALL_FOLDS), which recompute each
 *                 fold's part from its rows;
 *                 otherwise they may be NULL.
 *   flags, ddof, XTX, XTY, mean_out, std_out, stream  as cv_products.
 *
 * Errors: CV_ERR_INVALID_ARG (null plan, no cv_products yet, bad flags /
 * ddof, inputs missing on a small-fold plan), CV_ERR_NOT_SCALABLE,
 * CV_ERR_CUDA.  Does not allocate or synchronise.
 */
cv_status cv_finalize(cv_plan_t plan, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                      int flags, int ddof, void *XTX, void *XTY,
                      double *mean_out, double *std_out, void *stream);

/*
 * Fold sharding over several GPUs (one process per GPU).  The paper's Lemma 2
 * says the Gram over all rows is the sum of the folds' validation Grams, and
 * every fold's training products follow from that total and the fold's own
 * Gram (Algorithm 7 steps 8-9, 17-19; Propositions 7, 8, 15, 16).  So each
 * GPU can contract only the rows of the folds it owns, the GPUs sum their
 * partial totals once, and each GPU finishes its own folds:
 *
 *   plan  = cv_plan_ex(..., opts with fold_begin/fold_end = this GPU's folds)
 *   cv_products_partial(plan, X, Y, ex_int, ex_real, stream)
 *   all-reduce (sum) ex_int (int64) and ex_real (double) over the GPUs
 *   cv_finalize_total(plan, ex_int, ex_real, flags, ddof, XTX, XTY, ...)
 *
 * The exchange is independent of N and P: the upper block triangle of the
 * (K + M + 1)-column Gram in the contraction's units, in 128 x 128 tiles.
 * Every GPU passes the same full X and Y (it reads only its folds' rows and
 * the shift estimate's fixed sample of rows, so all GPUs shift and scale the
 * columns identically).
 *
 * cv_plan_exchange_size -- the lengths of the exchange buffers of a plan:
 * *n_int int64 values (0 on the FP64 path) and *n_real doubles.
 */
cv_status cv_plan_exchange_size(cv_plan_t plan, int64_t *n_int, int64_t *n_real);

/*
 * cv_products_partial -- the first half of a sharded cv_products: shift
 * estimate, operand conversion, contraction and fold sums over the plan's
 * folds, then this GPU's partial total written to the exchange buffers.
 *
 *   plan          a plan made with a fold range (cv_plan_options).
 *   X, ldx, Y, ldy  the full inputs, as cv_products.
 *   ex_int        device, int64[n_int] (may be NULL when n_int is 0): the
 *                 exact integer part of the split precisions' partial total.
 *   ex_real       device, double[n_real]: the rest of the partial total.
 *
 * Enqueued on `stream`; no synchronisation, no allocation.  Errors:
 * CV_ERR_INVALID_ARG (not a sharded plan, null buffers, bad inputs),
 * CV_ERR_CUDA.
 */
cv_status cv_products_partial(cv_plan_t plan, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                              int64_t *ex_int, double *ex_real, void *stream);

/*
 * cv_finalize_total -- the second half: takes the exchange buffers after the
 * element-wise sum over every GPU of the computation (the Gram over all
 * rows), then runs the statistics and the epilogue of the plan's folds.
 * Arguments after the buffers as cv_products; XTX, XTY, mean_out and std_out
 * hold fold_end - fold_begin folds.  Later cv_finalize calls on the plan
 * reuse the total for other flags.  Errors: CV_ERR_INVALID_ARG (not a
 * sharded plan, no cv_products_partial before, null buffers, bad flags or
 * ddof), CV_ERR_NOT_SCALABLE, CV_ERR_CUDA.
 */
cv_status cv_finalize_total(cv_plan_t plan, const int64_t *ex_int, const double *ex_real, int flags, int ddof,
                            void *XTX, void *XTY, double *mean_out, double *std_out, void *stream);

/*
 * Models on the products.  The paper names ridge regression and ordinary
 * least squares through the normal equations as consumers of X^T X and
 * X^T Y, and cross-validation as fitting on each training partition and
 * evaluating on its validation partition (Section 1).
 *
 * cv_ridge -- for every fold p, B_p = (XTX_p + lambda I)^-1 XTY_p, by the
 * Cholesky factorisation XTX_p + lambda I = L L^T in FP64 and forward / back
 * substitution (lambda = 0 is OLS).  The model lives in the space the
 * products were preprocessed into.
 *
 *   P, K, M       folds, X columns, Y columns (P >= 1, K >= 1, M >= 0).
 *   XTX, XTY      device, FP64, P x K x K and P x K x M row-major, as written
 *                 by cv_products with out_dtype CV_F64 (the full layout).
 *                 Only the lower triangle of each XTX_p is read.
 *   lambda        the ridge parameter (finite; negative values are allowed
 *                 and simply shift the diagonal).
 *   L             device scratch, P x K x K doubles, caller-owned; receives
 *                 each fold's factor L_p, row-major (L[p][i][j], j <= i),
 *                 strict upper triangle zero; partial when info[p] != 0.
 *   B             device output, P x K x M doubles (may be NULL when M = 0).
 *   info          device output, P int32: 0, or j + 1 when the pivot of
 *                 column j is not positive (XTX_p + lambda I is not positive
 *                 definite; B_p is then NaN).
 *
 * Blocked right-looking factorisation in 32 x 32 blocks, every fold's blocks
 * in the same launches (2 per block column), then one solve launch (a
 * cluster of 8 blocks per fold and chunk of responses); enqueued on
 * `stream`, no synchronisation, no allocation.  Errors: CV_ERR_INVALID_ARG,
 * CV_ERR_UNSUPPORTED (P > 65535, or K > 186880 with M > 0: one response's
 * right-hand sides must fit a block's shared memory), CV_ERR_CUDA.
 */
cv_status cv_ridge(int32_t P, int32_t K, int32_t M, const double *XTX, const double *XTY, double lambda,
                   double *L, double *B, int32_t *info, void *stream);

/*
 * cv_ridge_press -- the per-fold models' squared prediction error on each
 * validation partition: press[p][m] = sum over the validation rows n of fold
 * p of (y_nm - y^_nm)^2.  A validation row is preprocessed with its fold's
 * TRAINING statistics, x~_k = (x_k - [cX] mean_k) / ([sX] ? std_k : 1), so
 * nothing leaks from the validation partition; the prediction x~ B_p is
 * mapped back to Y's units: y^ = (x~ B_p) ([sY] ? std : 1) + ([cY] ? mean : 0).
 *
 *   plan          the plan of the products (its fold-sorted rows are used).
 *   X, ldx, Y, ldy  the inputs of that cv_products call (M >= 1).
 *   flags         the flags the products and B were made with.
 *   mean, std     device, P x (K + M) doubles: cv_products' mean_out and
 *                 std_out for those flags.
 *   B             device, P x K x M doubles from cv_ridge.
 *   press         device output, P x M doubles (zeroed, then accumulated
 *                 with atomic adds: the summation order is not fixed).
 *
 * Enqueued on `stream`; no synchronisation, no allocation.  Errors:
 * CV_ERR_INVALID_ARG (null pointers, M = 0, ld or flags out of range),
 * CV_ERR_UNSUPPORTED (a plan with a fold range, or K > 12795: one response's
 * model must fit a block's shared memory), CV_ERR_CUDA.
 */
cv_status cv_ridge_press(cv_plan_t plan, const void *X, int64_t ldx, const void *Y, int64_t ldy, int flags,
                         const double *mean, const double *std, const double *B, double *press, void *stream);

/*
 * cv_plan_status -- synchronise `stream` and return the first device-side
 * error recorded by this plan's cv_products calls (CV_OK if none), then clear
 * it.
 */
cv_status cv_plan_status(cv_plan_t plan, void *stream);

/*
 * cv_plan_fold_offsets -- copy the plan's fold boundaries (Algorithm 1) to
 * host memory: offsets[p] .. offsets[p+1] is fold p's range in the
 * fold-sorted row order; offsets has P + 1 entries.
 */
cv_status cv_plan_fold_offsets(cv_plan_t plan, int64_t *offsets);

/*
 * cv_plan_permutation -- copy the plan's fold-sorted row order (int32[N]) to
 * host memory: rows of fold p, increasing, at [offsets[p], offsets[p+1]).
 * Synchronises the plan's stream.
 */
cv_status cv_plan_permutation(cv_plan_t plan, int32_t *perm);

/* cv_plan_workspace_bytes -- device bytes owned by the plan. */
cv_status cv_plan_workspace_bytes(cv_plan_t plan, int64_t *bytes);

/*
 * Phases of one cv_products call, in the order they run on the stream:
 *   0 shift estimate       per-column shift and scale from a row sample
 *   1 operand conversion   split path only: W written once as FP16 hi/lo
 *                          tiles (zero time on the FP64 path)
 *   2 Gram contraction     per-segment tiles of W^T W (Alg. 7 steps 3, 8)
 *   3 fold sums            per-fold and total sums of the tiles (Lemma 2)
 *   4 fold statistics      training means, stds and epilogue factors
 *   5 epilogue             centred/scaled products written out
 */
#define CV_NUM_PHASES 6

/*
 * cv_plan_profile -- turn per-phase timing of cv_products on (enable != 0)
 * or off, and reset the accumulated times.  While on, every cv_products call
 * records CUDA events on its stream at the boundaries of its CV_NUM_PHASES
 * phases, for at most 4096 calls until the next reset.  Events come from a
 * pool created here; no call allocates afterwards.
 */
cv_status cv_plan_profile(cv_plan_t plan, int enable);

/*
 * cv_plan_phase_ms -- synchronise on the last recorded event and return, in
 * ms[0 .. CV_NUM_PHASES-1], the summed device time of each phase over the
 * calls recorded since cv_plan_profile, and in *calls their number.
 */
cv_status cv_plan_phase_ms(cv_plan_t plan, double *ms, int32_t *calls);

/*
 * cv_plan_launches -- the number of GPU kernels that cv_products and
 * cv_finalize calls on this plan have enqueued since the plan was made
 * (cv_plan's own launches are not counted).  Host-only; does not synchronise.
 */
cv_status cv_plan_launches(cv_plan_t plan, int64_t *count);

/*
 * Batches of independent problems (many small cross-validations at once).
 * The paper has no counterpart: this is a throughput interface for many
 * problems, each computed exactly as cv_products computes it for a plan made
 * with the options cv_batch_plan_options reports.
 *
 * cv_problem describes one problem: its shape, fold ids, inputs, flags and
 * outputs, with the meaning, layout and ownership of the same arguments of
 * cv_plan and cv_products.  Y may be NULL when M == 0; XTX, XTY, mean_out
 * and std_out may be NULL to skip.
 */
typedef struct cv_problem {
    int64_t N;
    int32_t K, M, P;
    const int32_t *fold_ids;   /* int32[N] in [0, P) (device or host, see cv_batch_plan) */
    const void *X;             /* device, row-major N x K, leading dimension ldx */
    int64_t ldx;
    const void *Y;             /* device, row-major N x M, leading dimension ldy */
    int64_t ldy;
    int flags, ddof;           /* as cv_products */
    void *XTX, *XTY;           /* device outputs, P x K x K and P x K x M */
    double *mean_out, *std_out;   /* optional device outputs, P x (K + M) */
} cv_problem;

typedef struct cv_batch_s *cv_batch_t;

/*
 * cv_batch_plan -- cv_plan for each of `count` problems, all with the same
 * in_dtype, out_dtype and precision.  Only the shape and fold_ids of each
 * cv_problem are read.  Synchronises `stream` once per problem.  Errors as
 * cv_plan for any problem (nothing is leaked; *out is NULL), and
 * CV_ERR_INVALID_ARG for count < 1.
 *
 * A batch whose precision resolves to a tensor-core split precision
 * (CV_PREC_FP16X3, CV_PREC_BF16X3, CV_PREC_TF32, CV_PREC_TF32X3), with in_dtype == CV_F32 and
 * P <= 32 in every problem, runs as batched launches: each of the path's five
 * stages is one kernel launch over all problems' work units (the last one
 * per class of fold counts present, P <= 8, <= 16, <= 32), and every problem
 * is planned with the fold-grouped strategy (never the small-fold one),
 * whatever its fold sizes, and with its share of the device's SMs (in
 * proportion to its rows times Gram tiles, at least 1) as the plan's ctas.
 * The work tables (about 16 bytes per work unit) are built here and stay on
 * the device with the batch.  Any other
 * batch runs as a CUDA graph of the problems' own cv_products calls.
 */
cv_status cv_batch_plan(cv_batch_t *out, const cv_problem *probs, int32_t count, int fold_ids_on_device,
                        cv_dtype in_dtype, cv_dtype out_dtype, cv_precision prec, void *stream);

/*
 * cv_batch_products -- cv_products for every problem of the batch, enqueued
 * on `stream`.  probs[i] must have the shape problem i had in cv_batch_plan;
 * its inputs, outputs, flags and ddof may differ from call to call.
 *
 * Batched launches (see cv_batch_plan): five to seven kernels on `stream`.
 * For batches of at most 256 problems the problems' pointers, flags and ddof
 * travel as kernel parameters: the call copies nothing to the device and
 * waits for nothing on the host, so it can be captured into a CUDA graph
 * (whose replays use the arguments of the captured call).  Larger batches
 * copy them to the device (from pinned staging the batch owns) when they
 * differ from the previous call's, waiting for the previous copy before
 * rewriting the staging: such a call is not capturable.  Results are bitwise
 * those of the problem's own fold-grouped plan through cv_products.
 *
 * CUDA graph: one graph whose branches run the problems' cv_products
 * concurrently on the batch's internal streams; captured on the first call
 * and re-captured only when a descriptor changes, so a repeated call costs
 * one graph launch.
 *
 * Calls on one batch share its plans' workspaces and its device copy of the
 * arguments, so they must not overlap on the device: issue them on one
 * stream, or order them with events.
 *
 * Does not synchronise otherwise.  Errors: CV_ERR_INVALID_ARG (a shape
 * differs, or an argument cv_products would reject), CV_ERR_NOT_SCALABLE,
 * CV_ERR_CUDA.  Device-side errors are returned by cv_batch_status.
 */
cv_status cv_batch_products(cv_batch_t batch, const cv_problem *probs, void *stream);

/* cv_batch_status -- cv_plan_status over every problem of the batch: the
 * first device-side error found, CV_OK if none; synchronises `stream`. */
cv_status cv_batch_status(cv_batch_t batch, void *stream);

/* cv_batch_plan_options -- the options problem `index` of the batch was
 * planned with: a cv_plan_ex with these options, the problem's shape, fold
 * ids, dtypes and precision gives a plan whose cv_products results are
 * bitwise those of the batch.  CV_ERR_INVALID_ARG for an index out of range. */
cv_status cv_batch_plan_options(cv_batch_t batch, int32_t index, cv_plan_options *opts);

/* cv_batch_launches -- the number of GPU kernels cv_batch_products calls on
 * this batch have enqueued (for batched launches 4 per call plus one per
 * class of fold counts present, P <= 8, <= 16, <= 32; for a graph, the
 * kernels of its captured cv_products calls), and in *batched (may be NULL)
 * 1 if the batch runs as batched launches, 0 if as a graph.  Host-only. */
cv_status cv_batch_launches(cv_batch_t batch, int64_t *count, int32_t *batched);

/* cv_batch_destroy -- release the plans, streams, tables and graph of a
 * batch.  Work already enqueued with it must have completed. */
cv_status cv_batch_destroy(cv_batch_t batch);

/*
 * cv_products_batched -- one-shot batch: cv_batch_plan, cv_batch_products,
 * cv_batch_status and cv_batch_destroy in one call; fold ids on the device.
 * Synchronises `stream` before returning.
 */
cv_status cv_products_batched(const cv_problem *probs, int32_t count, cv_dtype in_dtype,
                              cv_dtype out_dtype, cv_precision prec, void *stream);

/*
 * cv_products_f64_static -- the CV_PREC_FP64 products of cv_products for a
 * small problem, in one call that allocates no memory at all.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory, such as code running in a process whose GPU
 * memory another framework's allocator owns under a fixed budget, or a
 * latency-critical loop where a cudaMalloc (which can synchronize the device
 * and can fail under memory pressure) is not acceptable.
 *
 * Instead of a plan's workspace it uses one scratch array of about 11 MB that
 * the library declares in device memory; every GPU that loads the library
 * holds that array until the process exits.  Its device address is looked up
 * (cudaGetSymbolAddress) on the first call made on each device, with that
 * device current; make that first call before any stream capture.
 *
 * Arguments are those of cv_plan and cv_products together: fold_ids is a
 * device pointer (int32[N], values in [0, P)); X, Y, the outputs and the
 * optional mean_out / std_out follow cv_products; in_dtype / out_dtype as in
 * cv_plan.  The call synchronizes `stream` twice (once to read the fold sizes
 * back, once after copying its host-side tables to the device), then enqueues
 * the rest and returns without waiting.  Because it synchronizes, it must not
 * be called while `stream` is being captured into a CUDA graph.
 *
 * Limits: N <= 32768, K + M + 1 <= 128, 2 <= P <= 16.  Larger problems return
 * CV_ERR_UNSUPPORTED (use cv_plan / cv_products).  Other errors as cv_plan and
 * cv_products.
 *
 * All calls share the one scratch array and each call overwrites what the
 * previous one left there: calls whose device work overlaps (on different
 * streams, or from different host threads on one device) race and give wrong
 * results.  Serialize them, for example on one stream.
 */
cv_status cv_products_f64_static(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *fold_ids,
                                 const void *X, int64_t ldx, const void *Y, int64_t ldy,
                                 cv_dtype in_dtype, cv_dtype out_dtype, int flags, int ddof,
                                 void *XTX, void *XTY, double *mean_out, double *std_out,
                                 void *stream);

/* cv_plan_destroy -- free the plan and its workspace; NULL is a no-op.
 * Work already enqueued with this plan must have completed. */
cv_status cv_plan_destroy(cv_plan_t plan);

/* cv_status_string -- static, human-readable name of a status code. */
const char *cv_status_string(cv_status s);

#ifdef __cplusplus
}
#endif

#endif /* CVX_H */
