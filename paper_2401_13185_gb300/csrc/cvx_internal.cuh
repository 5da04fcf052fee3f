// cvx_internal.cuh -- plan layout and kernel entry points shared by the
// translation units of the CUDA library (not part of the public ABI).
//
// Data model.  W = [X' | Y' | 1] is the N x D matrix (D = K + M + 1) of
// shifted (and, for split precision, power-of-two scaled) columns followed by
// a column of ones.  For every fold p the library forms the upper triangle of
// H_p = W_{V_p}^T W_{V_p}, which holds in one symmetric matrix:
//   * X_V'^T X_V'  and  X_V'^T Y_V'       (Algorithm 7 step 8),
//   * the diagonal of Y_V'^T Y_V'          (sums of squares, step 19),
//   * W'^T 1 = column sums of X' and Y'   (step 17),
//   * 1^T 1 = |V_p|.
// Row/column sums and sums of squares therefore come out of the same
// contraction as the Gram.  H is computed in 128 x 128 tiles (bi <= bj) over
// "segments": contiguous ranges of the fold-sorted row order that never
// straddle a fold.  Each (segment, tile) work item writes one FP64 partial
// tile; the stats and epilogue kernels reduce partials per fold and in total
// (Lemma 2: the training product is the total minus the validation part).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "../../include/cvx.h"

namespace cvx {

constexpr int TILE = 128;                 // rows/cols of one H tile
constexpr int TILE_ELEMS = TILE * TILE;   // FP64 values in one partial tile

struct Segment {          // rows [begin, end) of the fold-sorted order, all in `fold`
    int32_t begin, end, fold, pad;
};

struct TileCoord {
    int32_t bi, bj;       // block row / column of H, bi <= bj
};

// Split-precision operands: the fold-sorted rows are cut into k-blocks of
// OPS_KB rows inside one segment; every (k-block, 128-column block) pair
// holds its FP16 hi and lo tiles in the tensor core's shared-memory image.
constexpr int OPS_KB = 64;
constexpr int OPS_TILE_BYTES = 2 * TILE * OPS_KB * 2;   // hi + lo: 32 KB

// Split precisions of the tensor-core contraction (PlanView::kind).
enum : int {
    KIND_FP16X3 = 0,   // FP16 integer hi + FP16 lo, hi*hi exact in its own accumulator, 4 products
    KIND_BF16X3 = 1,   // BF16 hi + BF16 lo, hi*hi + hi*lo + lo*hi in one FP32 accumulator
    KIND_TF32 = 2,     // one TF32 product in one FP32 accumulator
    KIND_TF32X3 = 3    // TF32 hi + TF32 lo, hi*hi + hi*lo + lo*hi in FP32 accumulators
};

// Bytes of one (k-block, column block) operand tile of a precision.  TF32X3
// keeps, for each 32-row half of the k-block, a 16 KB hi tile then a 16 KB
// lo tile (the layout of one FP16 k-block), so its tiles are twice as large.
__host__ __device__ constexpr int ops_tile_bytes(int kind) {
    return kind == KIND_TF32X3 ? 2 * OPS_TILE_BYTES : OPS_TILE_BYTES;
}

struct KBlock {
    int32_t row0;         // first row in the fold-sorted order
    int32_t valid;        // rows in use (<= OPS_KB); the rest are zero
};

// Device error word bits (OR-ed by kernels, read by cv_plan_status).
enum : int { DEV_ERR_RANGE = 1, DEV_ERR_TIMEOUT = 2 };

struct ShiftParams {       // per W column c, 0 <= c < D
    double *shift;         // s_c subtracted before the contraction (0 for ones)
    double *inv_scale;     // 2^-e_c, undoes the split path's scaling
    float *shift_f;        // s_c as float (FP32 inputs: exactly s_c)
    float *scale_f;        // 2^e_c as float
};

// Programmatic dependent launch.  Every kernel of the library is launched
// with programmatic stream serialization, so that it is scheduled while its
// predecessor on the stream drains, and starts with grid_dep_wait(), which
// returns once the predecessor grid has completed and its memory is visible.
// Because every kernel waits before its first global-memory access (and
// before any early exit), completion stays ordered along the whole stream.
// grid_dep_launch() lets the successor be scheduled before this grid ends.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace cvx

namespace cvx {

// Everything a kernel needs from a plan: plain data, passed by value.
struct PlanView {
    int64_t N;
    int32_t K, M, P, D, nb, ntiles, nsegs;
    int32_t int_bits;         // split precision: sampled column max scaled to 2^int_bits
    int32_t nlast;            // split precision: columns of the last 128-column block of W the
                              // contraction computes (its used columns rounded up to a multiple of
                              // 16, the MMA's N granularity); the others are never read
    int32_t nkb;              // split precision: number of k-blocks
    KBlock *kblocks;          // nkb
    int32_t *seg_kb;          // nsegs + 1: first k-block of each segment
    void *ops;                // nkb * nb * OPS_TILE_BYTES split operand tiles
    int32_t *perm;            // N: fold-sorted row order
    int64_t *offs;            // P + 1 fold boundaries in that order
    Segment *segs;            // nsegs
    int32_t *fold_seg;        // P + 1: first segment of each fold
    TileCoord *tiles;         // ntiles
    double *partials;         // nsegs * ntiles * TILE_ELEMS partial tiles of H, item (seg,
                              // tile) at seg * ntiles + tile, each tile column-major:
                              // (li, lj) at lj * TILE + li.  FP64 path: doubles.  Split
                              // path: the same bytes hold an int32 array (exact hi * hi
                              // sums) followed by a float array (cross terms), see
                              // part_hi / part_lo.
    int32_t split;            // 1 when the partials use the split layout
    int32_t kind;             // split precision (KIND_*): its operand image and products
    int32_t small;            // 1: small-fold strategy (segments ignore folds, only the total
                              // of H is reduced; each fold's part is recomputed from its rows)
    void *fold_sq;            // small-fold strategy: P * (K + M) {sum, sum of squares} of each
                              // fold's rows in contraction units (float2 split, double2 FP64)
    void *gfold;              // FP64 path: P * ntiles * TILE_ELEMS, H of each fold's rows (column-major tiles)
    void *gtot;               // ntiles * TILE_ELEMS: H over all rows
                              // FP64 path: doubles.  Split path: an int64 array (exact hi * hi
                              // sums) followed by a float array (cross terms).
    ShiftParams sp;
    double *stats;            // P * (K + M) * 4: per fold and column {A, B, C, E}, see k_fold_stats
    float4 *fac_f;            // split path: P * (K + M) factors {A, B, C, E} / 2^t, see k_fold_stats
    int32_t *fac_t;           // split path: P * (K + M) exponents t of those factors
    int32_t nsample;          // rows in the shift estimate's strided sample: row k N / nsample
    int32_t p_lo, p_hi;       // folds the plan computes outputs for: [p_lo, p_hi) (all: 0, P);
                              // outputs and mean/std hold fold p at index p - p_lo
    int32_t packed;           // 1: X^T X written as each fold's upper triangle, row by row
    uint64_t wait_ns;         // bound of every wait inside the tensor-core kernels
    int *err;                 // device error word
};

// Offset of entry (i, j), i <= j, in a fold's packed upper triangle of K x K.
__host__ __device__ inline int64_t packed_upper(int K, int i, int j) {
    return (int64_t)i * K - (int64_t)i * (i - 1) / 2 + (j - i);
}

// Values per fold of the X^T X output of a plan view.
__host__ __device__ inline int64_t xtx_fold_elems(const PlanView &v) {
    return v.packed ? (int64_t)v.K * (v.K + 1) / 2 : (int64_t)v.K * v.K;
}

}  // namespace cvx

namespace cvx {

// Batched launches: every problem of a batch keeps its plan, and each stage
// of the path runs as ONE launch over all problems' work units.
struct ProblemArgs {           // the per-call arguments of one problem
    const void *X, *Y;
    int64_t ldx, ldy;
    void *XTX, *XTY;
    double *mean_out, *std_out;
    int32_t flags, ddof, x_vec, pad;
};

// A call's per-problem arguments as a kernel parameter (CUDA 12.1+ allows
// kernel parameters up to 32 KB): nothing is copied to the device per call,
// so a call can be captured into a CUDA graph.  Larger batches keep their
// arguments in device memory (BatchTables::args).
constexpr int BATCH_ARGS_MAX = 256;
struct BatchArgs {
    ProblemArgs a[BATCH_ARGS_MAX];
};

struct BatchTables {           // device tables built by cv_batch_plan
    const PlanView *views;     // [count] the plans
    const ProblemArgs *args;   // [count] this call's arguments in device memory, or null: in BatchArgs
    const int2 *shift_units;   // (problem, column group of 32): one cluster each
    int32_t n_shift;
    const int4 *conv_units;    // (problem, k-block begin, end, -): one block each
    int32_t n_conv;
    const int2 *gram_items;    // (problem, work item), grouped by CTA
    const int32_t *gram_cta;   // [gram_ctas + 1] each CTA's range of gram_items
    int32_t gram_ctas;
    const int4 *stats_units;   // (problem, first column, fold, -): one 32-thread block each
    int32_t n_stats;
    const int4 *epi_units;     // (problem, tile, 16 x 16 sub-tile, fold-count class): one block each
    int32_t n_epi;
    int32_t max_P, kind, out_f64;
};

__device__ __forceinline__ const ProblemArgs &batch_arg(const BatchTables &bt, const BatchArgs &ba, int i) {
    return bt.args ? bt.args[i] : ba.a[i];
}

}  // namespace cvx

struct cv_plan_s {
    cvx::PlanView v;
    cv_dtype in_dtype, out_dtype;
    cv_precision prec;
    int device, num_sms;
    cv_plan_options opts;                      // as given to cv_plan_ex (defaults for cv_plan)
    std::vector<int64_t> h_offs;              // P + 1 fold boundaries
    std::vector<cvx::Segment> h_segs;
    void *d_block;                             // one device allocation, carved
    size_t ws_bytes;
    float *ypack;                              // split path, FP32 inputs: N x ypack_width [Y | 1 | 0 ..]
    int ypack_width;
    // phase timing (cv_plan_profile): CV_NUM_PHASES + 1 events per recorded call
    bool profiling;
    int prof_calls;
    std::vector<cudaEvent_t> prof_events;
    // kernels enqueued by cv_products / cv_finalize on this plan since it was made
    mutable int64_t launches;
    // a cv_products call has been enqueued: the fold sums cv_finalize reuses exist
    bool has_sums;
    // the plan owns a fold range (cv_plan_options fold_begin / fold_end): it
    // runs as cv_products_partial + cv_finalize_total
    bool sharded;
    // the fold-sorted order is mostly gathered rows (not runs of consecutive
    // rows): the split conversion copies whole rows
    bool gathered;
    // a cv_products_partial call has been enqueued on a sharded plan
    bool has_partial;
};

namespace cvx {

// fold_sort.cu
cudaError_t fold_count(const int32_t *folds, int64_t N, int32_t P,
                       unsigned long long *counts, int *bad, cudaStream_t st);
cudaError_t fold_sort(const int32_t *folds, int64_t N, int32_t P, int32_t *perm,
                      void *tmp, size_t tmp_bytes, cudaStream_t st);
// Rows per block of the fold sort's radix passes, and the scratch the sort
// needs for N rows: two key buffers, two value buffers and one 256-bin
// histogram per block.
constexpr int FOLD_SORT_ROWS_PER_BLOCK = 4096;
constexpr size_t fold_sort_tmp_bytes_for(int64_t N) {
    return (size_t)N * sizeof(int32_t) * 4 +
           (size_t)((N + FOLD_SORT_ROWS_PER_BLOCK - 1) / FOLD_SORT_ROWS_PER_BLOCK) * 256 * sizeof(unsigned int) +
           1024;
}
size_t fold_sort_tmp_bytes(int64_t N);
// adds to *breaks the number of n with perm[n + 1] != perm[n] + 1
cudaError_t perm_breaks(const int32_t *perm, int64_t N, unsigned long long *breaks, cudaStream_t st);

// stats_epilogue.cu
cudaError_t shift_estimate(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y,
                           int64_t ldy, bool split, cudaStream_t st);
cudaError_t fold_sums(const cv_plan_s *pl, cudaStream_t st);
cudaError_t fold_stats(const cv_plan_s *pl, int flags, int ddof, double *mean_out, double *std_out,
                       cudaStream_t st);
constexpr int SHIFT_SAMPLE = 1024;   // rows in the shift estimate's strided sample
constexpr int SHIFT_ROWS_PER_CHUNK = 128;
cudaError_t epilogue(const cv_plan_s *pl, int flags, void *XTX, void *XTY, cudaStream_t st);
// split path, fold-grouped strategy, few folds: statistics straight from the
// segment partials and one fold-sum + epilogue pass (no fold-sum kernel)
bool fused_tail(const cv_plan_s *pl);
cudaError_t split_stats(const cv_plan_s *pl, int flags, int ddof, double *mean_out, double *std_out, cudaStream_t st);
cudaError_t fold_epilogue_split(const cv_plan_s *pl, int flags, void *XTX, void *XTY, cudaStream_t st);

// batched stages (one launch each over every problem of a batch)
cudaError_t shift_estimate_batched(const BatchTables &bt, const BatchArgs &ba, cudaStream_t st);
cudaError_t convert_batched(const BatchTables &bt, const BatchArgs &ba, cudaStream_t st);
cudaError_t gram_tc_batched(const BatchTables &bt, cudaStream_t st);
cudaError_t split_stats_batched(const BatchTables &bt, const BatchArgs &ba, cudaStream_t st);
cudaError_t fold_epilogue_split_batched(const BatchTables &bt, const BatchArgs &ba, cudaStream_t st);
constexpr int BATCH_FOLD_MAX = 32;   // folds per problem the batched tail takes

// api.cu: the shape of a problem's work decomposition in units of its
// contraction (rows times upper-triangle tiles of 128 x 128)
int64_t plan_work_units(int64_t N, int32_t K, int32_t M);

// api.cu: the argument checks of cv_products (CV_OK when the call may proceed)
cv_status products_arg_status(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                              int flags, int ddof);
// api.cu: flags, ddof and Definition 6's scalability check alone
cv_status flags_arg_status(const cv_plan_s *pl, int flags, int ddof);
// api.cu: CUDA error -> library status
cv_status status_of(cudaError_t e);

// shard.cu: the partial total of the contraction to / from the exchange buffers
cudaError_t export_total(const cv_plan_s *pl, long long *ex_int, double *ex_real, cudaStream_t st);
cudaError_t import_total(const cv_plan_s *pl, const long long *ex_int, const double *ex_real, cudaStream_t st);

// small_folds.cu (small-fold strategy)
cudaError_t small_fold_colsums(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                               cudaStream_t st);
cudaError_t small_fold_epilogue(const cv_plan_s *pl, int flags, const void *X, int64_t ldx, const void *Y,
                                int64_t ldy, void *XTX, void *XTY, cudaStream_t st);

// gram_f64.cu
cudaError_t gram_f64(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y,
                     int64_t ldy, cudaStream_t st);

// gram_tc.cu
cudaError_t convert_split(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y,
                          int64_t ldy, cudaStream_t st);
cudaError_t gram_tc(const cv_plan_s *pl, cudaStream_t st);

// Split-path partial arrays carved from PlanView::partials.
__host__ __device__ inline int32_t *part_hi(const PlanView &v) { return reinterpret_cast<int32_t *>(v.partials); }
__host__ __device__ inline float *part_lo(const PlanView &v) {
    return reinterpret_cast<float *>(v.partials) + (int64_t)v.nsegs * v.ntiles * TILE_ELEMS;
}

// Split path: fold p's sum H_p at element it (= tile * TILE_ELEMS + e) of the
// tiles, from the partials of the fold's own segments in segment order: the
// hi * hi parts exactly in int64, the cross terms in FP32.  (The fold-grouped
// strategy's segments never straddle a fold; a fold holds a few of them.)
__device__ inline void fold_sum_split(const PlanView &v, int p, int64_t it, long long &hi, float &lo) {
    const int64_t seg_stride = (int64_t)v.ntiles * TILE_ELEMS;
    const int32_t *h = part_hi(v) + it;
    const float *l = part_lo(v) + it;
    hi = 0;
    lo = 0.0f;
    for (int g = v.fold_seg[p]; g < v.fold_seg[p + 1]; ++g) {
        hi += h[(int64_t)g * seg_stride];
        lo += l[(int64_t)g * seg_stride];
    }
}

// Training Gram entry G_T = H_R - H_p (Lemmas 2, 3) of fold p at element e of
// tile `tile`, in the contraction's (scaled, shifted) units.
__device__ inline double g_train(const PlanView &v, int p, int tile, int e) {
    const int64_t nt = (int64_t)v.ntiles * TILE_ELEMS;
    const int64_t it = (int64_t)tile * TILE_ELEMS + e;
    const int64_t ip = (int64_t)p * nt + it;
    if (v.split) {
        const long long *tot_hi = reinterpret_cast<const long long *>(v.gtot);
        const float *tot_lo = reinterpret_cast<const float *>(tot_hi + nt);
        long long fh;
        float fl;
        fold_sum_split(v, p, it, fh, fl);
        return (double)(tot_hi[it] - fh) + (double)(tot_lo[it] - fl);
    }
    return reinterpret_cast<const double *>(v.gtot)[it] - reinterpret_cast<const double *>(v.gfold)[ip];
}

// Entry e of tile `tile` of H over all rows, in the contraction's units.
__device__ inline double g_total(const PlanView &v, int tile, int e) {
    const int64_t nt = (int64_t)v.ntiles * TILE_ELEMS;
    const int64_t it = (int64_t)tile * TILE_ELEMS + e;
    if (v.split) {
        const long long *tot_hi = reinterpret_cast<const long long *>(v.gtot);
        const float *tot_lo = reinterpret_cast<const float *>(tot_hi + nt);
        return (double)tot_hi[it] + (double)tot_lo[it];
    }
    return reinterpret_cast<const double *>(v.gtot)[it];
}

// int64 -> FP32 without conversion instructions (profiles of the epilogue
// showed the integer-to-float conversions keeping this part's slow FP64 pipe
// busy).  |d| = a2 2^42 + a1 2^21 + a0 with 21-bit pieces; each piece becomes
// an exact float by placing it in the mantissa of 2^23 and subtracting 2^23,
// and two fused multiply-adds of non-negative terms join them: at most one
// rounding more than a correctly rounded conversion.
__host__ __device__ __forceinline__ float u21_to_float(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(0x4B000000u | x) - 8388608.0f;
#else
    union { uint32_t u; float f; } c;
    c.u = 0x4B000000u | x;
    return c.f - 8388608.0f;
#endif
}

__host__ __device__ __forceinline__ float ll_to_float(long long d) {
    const bool neg = d < 0;
    const unsigned long long a = neg ? 0ull - (unsigned long long)d : (unsigned long long)d;
    const float f0 = u21_to_float((uint32_t)a & 0x1FFFFFu);
    const float f1 = u21_to_float((uint32_t)(a >> 21) & 0x1FFFFFu);
    const float f2 = u21_to_float((uint32_t)(a >> 42) & 0x1FFFFFu);
    const float f = fmaf(f2, 4398046511104.0f, fmaf(f1, 2097152.0f, f0));
    return neg ? -f : f;
}

// Value of output entry (i, j) of fold p (i < K, i <= j < K + M) from the
// training Gram entry g in contraction units:
//   G'_T = G'_R - G'_p                                (Lemmas 2, 3)
//   centered:   v = G'_T - S'_T,i S'_T,j / N_T        (Propositions 7, 8;
//               X^T Y is centered when X or Y is, Lemma 9 / Table 1)
//   uncentered: v = G'_T + s_i S'_T,j + S'_T,i s_j + N_T s_i s_j
//               (expanding (x' + s_i)(z' + s_j) over T)
//   scaled:     v /= sigma_i sigma_j                   (Propositions 15, 16)
// evaluated with the per-column factors {A, B, C, E} of the fold statistics:
// G A_i A_j - B_i C_j, or G A_i A_j + E_i B_j + B_i E_j + N_T E_i E_j.
__device__ __forceinline__ double entry_f64(const PlanView &pl, bool centered, int p, int i, int j, double g) {
    const int KM = pl.K + pl.M;
    const double *fi = pl.stats + 4 * ((int64_t)p * KM + i);
    const double *fj = pl.stats + 4 * ((int64_t)p * KM + j);
    const double aa = fi[0] * fj[0];
    if (centered) return fma(g, aa, -fi[1] * fj[2]);
    const double nt = (double)(pl.N - (pl.offs[p + 1] - pl.offs[p]));
    return fma(g, aa, fma(fi[3], fj[1], fma(fi[1], fj[3], nt * fi[3] * fj[3])));
}

// r * 2^t as an FP64 value, exactly: the exponent is moved into FP64's range
// with integer operations (FP64 arithmetic is slow on this part); zeros,
// subnormals, non-finite values and results outside FP64's normal range take
// ldexp.
static __device__ __noinline__ double pow2_widen_slow(float r, int t) { return ldexp((double)r, t); }

__device__ __forceinline__ double pow2_widen(float r, int t) {
    const uint32_t b = __float_as_uint(r);
    const int ex = (int)((b >> 23) & 0xFFu);
    const int nex = ex - 127 + 1023 + t;
    if (ex != 0 && ex != 255 && nex > 0 && nex < 2047) {
        const unsigned long long d = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)nex << 52) |
                                     ((unsigned long long)(b & 0x7FFFFFu) << 29);
        return __longlong_as_double((long long)d);
    }
    return pow2_widen_slow(r, t);   // zeros, subnormals, non-finite: out of line
}

// 2^t as an FP64 value for -1022 <= t <= 1023 (exact, integer operations only).
__device__ __forceinline__ double pow2i(int t) {
    return __longlong_as_double((long long)(t + 1023) << 52);
}

// floor(log2 |x|) of a normal FP64 value from its exponent field.
__device__ __forceinline__ int ilogb_normal(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7FF) - 1023;
}

// Split path: the same formulas in FP32 on the factors normalised by 2^t per
// column (the split contraction carries about 22 significant bits, so FP32
// here adds rounding of the same order), widened to FP64 with the exact power
// of two 2^(t_i + t_j).
// The formulas on given factors: fi / fj = {A, B, C, E} / 2^t of columns i and
// j, t = t_i + t_j, ntr = N_T (uncentered only).
__device__ __forceinline__ double entry_split_f(bool centered, const float4 &fi, const float4 &fj, int t, float ntr,
                                                float g) {
    const float aa = fi.x * fj.x;
    float r;
    if (centered)
        r = fmaf(g, aa, -fi.y * fj.z);
    else
        r = fmaf(g, aa, fmaf(fi.w, fj.y, fmaf(fi.y, fj.w, ntr * fi.w * fj.w)));
    return pow2_widen(r, t);
}

__device__ __forceinline__ double entry_split(const PlanView &pl, bool centered, int p, int i, int j, float g) {
    const int KM = pl.K + pl.M;
    const float4 fi = pl.fac_f[(int64_t)p * KM + i];
    const float4 fj = pl.fac_f[(int64_t)p * KM + j];
    const int t = pl.fac_t[(int64_t)p * KM + i] + pl.fac_t[(int64_t)p * KM + j];
    const float ntr = centered ? 0.0f : ll_to_float(pl.N - (pl.offs[p + 1] - pl.offs[p]));
    return entry_split_f(centered, fi, fj, t, ntr, g);
}

__device__ __forceinline__ void st_f64x4(double *p, const double (&v)[4]) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(__double2loint(v[0])),
                 "r"(__double2hiint(v[0])), "r"(__double2loint(v[1])), "r"(__double2hiint(v[1])),
                 "r"(__double2loint(v[2])), "r"(__double2hiint(v[2])), "r"(__double2loint(v[3])),
                 "r"(__double2hiint(v[3]))
                 : "memory");
}

// Four consecutive output values at p (16- or 32-byte aligned when vec).
template <typename TOut>
__device__ __forceinline__ void store4(TOut *p, const TOut (&v)[4], bool vec, const bool (&ok)[4]) {
    if (vec) {
        if constexpr (sizeof(TOut) == 8)
            st_f64x4(reinterpret_cast<double *>(p), reinterpret_cast<const double(&)[4]>(v));
        else
            *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (ok[u]) p[u] = v[u];
    }
}

// r 2^t in the output type: FP64 exactly (pow2_widen); FP32 by moving the
// exponent when the result is a normal float (the same value as rounding
// the FP64 result), else through FP64.
template <typename TOut>
__device__ __forceinline__ TOut scaled_out(float r, int t) {
    if constexpr (sizeof(TOut) == 8) {
        return pow2_widen(r, t);
    } else {
        const uint32_t bits = __float_as_uint(r);
        const int ex = (int)((bits >> 23) & 0xFFu) + t;
        if (((bits >> 23) & 0xFFu) != 0u && ((bits >> 23) & 0xFFu) != 0xFFu && ex > 0 && ex < 255)
            return __uint_as_float((bits & 0x807FFFFFu) | ((uint32_t)ex << 23));
        return (float)pow2_widen(r, t);
    }
}

// Whole-row conversion (k_convert_direct, k_convert_batched): a block takes
// a run of k-blocks of about CD_PAIRS (16-row group, column) pairs, at most
// CD_MAX_RUN k-blocks.
constexpr int CD_PAIRS = 8192;
constexpr int CD_MAX_RUN = 64;

__host__ __device__ constexpr int direct_run(int D) {
    return D >= CD_PAIRS / 4 ? 1 : (CD_PAIRS / 4 / D < CD_MAX_RUN ? CD_PAIRS / 4 / D : CD_MAX_RUN);
}

__host__ __device__ inline int tile_index(int nb, int bi, int bj) {
    // row-major enumeration of the upper block triangle
    return bi * nb - (bi * (bi - 1)) / 2 + (bj - bi);
}

}  // namespace cvx
