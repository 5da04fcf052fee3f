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

// Device error word bits (OR-ed by kernels, read by cv_plan_status).
enum : int { DEV_ERR_RANGE = 1, DEV_ERR_TIMEOUT = 2 };

struct ShiftParams {       // per W column c, 0 <= c < D
    double *shift;         // s_c subtracted before the contraction (0 for ones)
    double *inv_scale;     // 2^-e_c, undoes the split path's scaling
    float *shift_f;        // s_c as float (FP32 inputs: exactly s_c)
    float *scale_f;        // 2^e_c as float
};

}  // namespace cvx

namespace cvx {

// Everything a kernel needs from a plan: plain data, passed by value.
struct PlanView {
    int64_t N;
    int32_t K, M, P, D, nb, ntiles, nsegs;
    int32_t int_bits;         // split precision: sampled column max scaled to 2^int_bits
    int32_t *perm;            // N: fold-sorted row order
    int64_t *offs;            // P + 1 fold boundaries in that order
    Segment *segs;            // nsegs
    int32_t *fold_seg;        // P + 1: first segment of each fold
    TileCoord *tiles;         // ntiles
    double *partials;         // nsegs * ntiles * TILE_ELEMS, FP64 partial tiles of H,
                              // item (seg, tile) at seg * ntiles + tile, each tile
                              // column-major: (li, lj) at lj * TILE + li
    double *gfold;            // P * ntiles * TILE_ELEMS: H of each fold's rows (column-major tiles)
    double *gtot;             // ntiles * TILE_ELEMS: H over all rows
    ShiftParams sp;
    double *stats;            // P * (K + M) * 2: {S'_T, sigma}
    int *err;                 // device error word
};

}  // namespace cvx

struct cv_plan_s {
    cvx::PlanView v;
    cv_dtype in_dtype, out_dtype;
    cv_precision prec;
    int device, num_sms;
    std::vector<int64_t> h_offs;              // P + 1 fold boundaries
    std::vector<cvx::Segment> h_segs;
    void *d_block;                             // one device allocation, carved
    size_t ws_bytes;
    // phase timing (cv_plan_profile): 5 events per recorded call
    bool profiling;
    int prof_calls;
    std::vector<cudaEvent_t> prof_events;
};

namespace cvx {

// fold_sort.cu
cudaError_t fold_count(const int32_t *folds, int64_t N, int32_t P,
                       unsigned long long *counts, int *bad, cudaStream_t st);
cudaError_t fold_sort(const int32_t *folds, int64_t N, int32_t P, int32_t *perm,
                      void *tmp, size_t tmp_bytes, cudaStream_t st);
size_t fold_sort_tmp_bytes(int64_t N);

// stats_epilogue.cu
cudaError_t shift_estimate(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y,
                           int64_t ldy, bool split, cudaStream_t st);
cudaError_t fold_stats(const cv_plan_s *pl, int ddof, double *mean_out, double *std_out,
                       cudaStream_t st);
cudaError_t epilogue(const cv_plan_s *pl, int flags, void *XTX, void *XTY, cudaStream_t st);

// gram_f64.cu
cudaError_t gram_f64(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y,
                     int64_t ldy, cudaStream_t st);

// gram_tc.cu
cudaError_t gram_tc(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y,
                    int64_t ldy, cudaStream_t st);

__host__ __device__ inline int tile_index(int nb, int bi, int bj) {
    // row-major enumeration of the upper block triangle
    return bi * nb - (bi * (bi - 1)) / 2 + (bj - bi);
}

}  // namespace cvx
