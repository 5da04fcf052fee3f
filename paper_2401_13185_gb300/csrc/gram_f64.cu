// gram_f64.cu -- FP64 CUDA-core contraction of the fold-grouped Gram.
//
// For every (segment, tile) work item the block forms the 128 x 128 tile
// (bi, bj) of W_S^T W_S over the segment's rows S (all in one fold), where
// W = [X - s | Y - s | 1] and the rows are gathered through the plan's
// fold-sorted order.  This is Algorithm 7 steps 8 (X_V^T X_V, X_V^T Y_V),
// 17 and 19 (validation sums and sums of squares, which sit in the ones
// column and on the diagonal of H) done in one pass with FP64 fused
// multiply-adds, the precision of the paper's own implementation (Section 7).
#include "cvx_internal.cuh"

namespace cvx {
namespace {

constexpr int KS = 8;        // rows per k-step
constexpr int THREADS = 256; // 16 x 16 threads, 8 x 8 outputs each

template <typename T>
__device__ __forceinline__ double w_value(const T *__restrict__ X, int64_t ldx,
                                          const T *__restrict__ Y, int64_t ldy, int K, int M,
                                          int64_t n, int c, const double *__restrict__ shift) {
    if (c < K) return (double)X[n * ldx + c] - shift[c];
    if (c < K + M) return (double)Y[n * ldy + (c - K)] - shift[c];
    if (c == K + M) return 1.0;
    return 0.0;
}

template <typename T>
__global__ void __launch_bounds__(THREADS) k_gram_f64(PlanView pl, const T *__restrict__ X, int64_t ldx,
                                                      const T *__restrict__ Y, int64_t ldy) {
    grid_dep_wait();
    grid_dep_launch();
    __shared__ double As[KS][TILE];
    __shared__ double Bs[KS][TILE];
    const int item = blockIdx.x;
    const int seg = item / pl.ntiles, tile = item % pl.ntiles;
    const Segment sg = pl.segs[seg];
    const TileCoord tc = pl.tiles[tile];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int K = pl.K, M = pl.M;
    const double *shift = pl.sp.shift;
    double acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;

    for (int r0 = sg.begin; r0 < sg.end; r0 += KS) {
#pragma unroll
        for (int q = 0; q < KS * TILE / THREADS; ++q) {
            const int idx = threadIdx.x + q * THREADS;
            const int kk = idx / TILE, c = idx % TILE;
            const int r = r0 + kk;
            double a = 0.0, b = 0.0;
            if (r < sg.end) {
                const int64_t n = pl.perm[r];
                a = w_value(X, ldx, Y, ldy, K, M, n, tc.bi * TILE + c, shift);
                b = w_value(X, ldx, Y, ldy, K, M, n, tc.bj * TILE + c, shift);
            }
            As[kk][c] = a;
            Bs[kk][c] = b;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            double av[8], bv[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) av[a] = As[k][ty * 8 + a];
#pragma unroll
            for (int b = 0; b < 8; ++b) bv[b] = Bs[k][tx * 8 + b];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
    // partial tiles are column-major: element (li, lj) at lj * TILE + li
    double *out = pl.partials + (int64_t)item * TILE_ELEMS;
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
        for (int a = 0; a < 8; a += 2)
            *reinterpret_cast<double2 *>(out + (tx * 8 + b) * TILE + ty * 8 + a) =
                make_double2(acc[a][b], acc[a + 1][b]);
}

}  // namespace

cudaError_t gram_f64(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                     cudaStream_t st) {
    const int64_t items = (int64_t)pl->v.nsegs * pl->v.ntiles;
    ++pl->launches;
    if (pl->in_dtype == CV_F32)
        return launch_pdl(k_gram_f64<float>, dim3((unsigned)items), dim3(THREADS), 0, st, pl->v, (const float *)X,
                          ldx, (const float *)Y, ldy);
    return launch_pdl(k_gram_f64<double>, dim3((unsigned)items), dim3(THREADS), 0, st, pl->v, (const double *)X, ldx,
                      (const double *)Y, ldy);
}

}  // namespace cvx
