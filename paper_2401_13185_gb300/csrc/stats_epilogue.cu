// stats_epilogue.cu -- column shift estimate, per-fold training statistics and
// the fused subtract / rank-one-correct / scale epilogue.
//
// Shift.  Every contraction works on x' = x - s_c with s_c the mean of a
// fixed strided sample of at most 4096 rows of column c.  Centered products
// and standard deviations are invariant to s (Propositions 7, 8: centering
// removes any constant), and uncentered products are recovered exactly from
// the shifted sums (see `epilogue`).  The shift keeps X'^T X' close to the
// centered product, so the |T| mean^T mean subtraction of Algorithm 7 step 15
// no longer cancels most of the digits when |mean| >> std.
//
// Statistics (Algorithm 7 steps 11-13, 17-24; Lemmas 7, 12-14).  From the
// per-segment partial tiles of H = W^T W (W = [X' | Y' | 1]) the kernel reads,
// per column c, the validation sums S'_V = H[c][ones] and sums of squares
// Q'_V = H[c][c], and forms the training sums S'_T = S'_R - S'_V and
// Q'_T = Q'_R - Q'_V (Lemma 14).  Then mean'_T = S'_T / N_T (Lemma 7 written
// with sums) and var = (Q'_T - S'_T mean'_T) / (N_T - ddof) (Lemma 12 after
// substituting the mean), clamped at 0; sigma = sqrt(var), replaced by 1 when
// var is 0 (step 24).
#include <math.h>

#include "cvx_internal.cuh"

namespace cvx {
namespace {

constexpr int SHIFT_SAMPLE = 1024;   // rows in the strided sample
constexpr int SHIFT_WARPS = 32;

// One block of 32 warps per 32 columns; lane = column, warp w takes sample
// rows w, w + 32, ... (row index k N / S), so every warp load is 32
// consecutive columns of one row, 32 loads in flight per thread.  The mean is
// formed as v_0 + mean(v - v_0) with v_0 the column's first sampled value, so
// a constant column gets exactly its constant as shift.  Partial sums are
// combined in a fixed order.  The second pass (maximum deviation) re-reads
// the same rows, which are cache-resident.
template <typename T>
__global__ void __launch_bounds__(SHIFT_WARPS * 32) k_shift_estimate(
    const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y, int64_t ldy, int64_t N, int K, int M,
    int S, bool split, int int_bits, ShiftParams sp) {
    constexpr int PER = SHIFT_SAMPLE / SHIFT_WARPS;
    __shared__ double red[SHIFT_WARPS][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const int D = K + M + 1;
    const bool live = c < K + M;
    // Branch-free column source: dead lanes read X[0][0] and are masked.
    const T *col = !live ? X : (c < K ? X + c : Y + (c - K));
    const int64_t ld = !live ? 0 : (c < K ? ldx : ldy);
    const double v0 = (double)col[0];
    T vals[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int k = warp + SHIFT_WARPS * j;
        const int64_t row = k < S ? ((int64_t)k * N) / S : 0;
        vals[j] = __ldg(col + row * ld);
    }
    double sum = 0.0;
#pragma unroll
    for (int j = 0; j < PER; ++j)
        if (warp + SHIFT_WARPS * j < S) sum += (double)vals[j] - v0;
    red[warp][lane] = sum;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < SHIFT_WARPS; ++w) s += red[w][lane];
    s = v0 + s / (double)S;
    if (sizeof(T) == 4) s = (double)(float)s;   // FP32 inputs: x - s exact in FP64
    __syncthreads();
    double mx = 0.0;
#pragma unroll
    for (int j = 0; j < PER; ++j)
        if (warp + SHIFT_WARPS * j < S) mx = fmax(mx, fabs((double)vals[j] - s));
    red[warp][lane] = mx;
    __syncthreads();
    if (warp == 0 && c < D) {
        double m = 0.0;
        for (int w = 0; w < SHIFT_WARPS; ++w) m = fmax(m, red[w][lane]);
        int e = 0;
        if (!live) {
            s = 0.0;   // the ones column
        } else if (split && m > 0.0) {
            int ex;
            frexp(m, &ex);          // m < 2^ex
            e = int_bits - ex;      // sampled max * 2^e < 2^int_bits
            e = max(-120, min(120, e));
        }
        sp.shift[c] = s;
        sp.shift_f[c] = (float)s;
        sp.scale_f[c] = ldexpf(1.0f, e);
        sp.inv_scale[c] = ldexp(1.0, -e);
    }
}

// Per-fold validation sums of H and the total over all rows (Lemma 2: the
// training product is the total minus the fold).  Thread per element of one
// tile; segments are visited once, in order, 8 loads in flight.
__global__ void __launch_bounds__(256) k_fold_reduce(PlanView pl) {
    const int tile = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const double *src = pl.partials + (int64_t)tile * TILE_ELEMS + e;
    const int64_t seg_stride = (int64_t)pl.ntiles * TILE_ELEMS;
    double tot = 0.0, acc = 0.0;
    int p = 0;
    int next_end = pl.fold_seg[1];
    constexpr int U = 8;
    for (int g0 = 0; g0 < pl.nsegs; g0 += U) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = g0 + u < pl.nsegs ? src[(int64_t)(g0 + u) * seg_stride] : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (g0 + u >= pl.nsegs) break;
            acc += v[u];
            if (g0 + u + 1 == next_end) {   // last segment of fold p
                pl.gfold[((int64_t)p * pl.ntiles + tile) * TILE_ELEMS + e] = acc;
                tot += acc;
                acc = 0.0;
                ++p;
                next_end = p < pl.P ? pl.fold_seg[p + 1] : -1;
            }
        }
    }
    pl.gtot[(int64_t)tile * TILE_ELEMS + e] = tot;
}

__device__ __forceinline__ double gfold_at(const PlanView &pl, int p, int tile, int e) {
    return pl.gfold[((int64_t)p * pl.ntiles + tile) * TILE_ELEMS + e];
}

// Thread per (fold p, column c < K + M).  stats[(p * (K+M) + c) * 2] = {S'_T, sigma}.
__global__ void k_fold_stats(PlanView pl, int ddof, double *__restrict__ mean_out,
                             double *__restrict__ std_out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    const int KM = pl.K + pl.M;
    if (c >= KM) return;
    const int ones = pl.D - 1;
    const int t_sum = tile_index(pl.nb, c / TILE, ones / TILE);
    const int e_sum = (ones % TILE) * TILE + (c % TILE);   // column-major tiles
    const int t_sq = tile_index(pl.nb, c / TILE, c / TILE);
    const int e_sq = (c % TILE) * TILE + (c % TILE);
    const double isc = pl.sp.inv_scale[c];
    const double s_all = pl.gtot[(int64_t)t_sum * TILE_ELEMS + e_sum];
    const double q_all = pl.gtot[(int64_t)t_sq * TILE_ELEMS + e_sq];
    const double s_v = gfold_at(pl, p, t_sum, e_sum);
    const double q_v = gfold_at(pl, p, t_sq, e_sq);
    const double nt = (double)(pl.N - (pl.offs[p + 1] - pl.offs[p]));
    const double st = (s_all - s_v) * isc;             // Lemma 14, shifted units
    const double qt = (q_all - q_v) * isc * isc;
    const double m = st / nt;                          // Lemma 7 via sums
    double var = nt - ddof > 0 ? (qt - st * m) / (nt - ddof) : NAN;
    if (var < 0.0) var = 0.0;                           // rounding below zero
    double sd = sqrt(var);
    if (var == 0.0) sd = 1.0;                           // Algorithm 7 step 24
    const int64_t o = (int64_t)p * KM + c;
    pl.stats[2 * o] = st;
    pl.stats[2 * o + 1] = sd;
    if (mean_out) mean_out[o] = pl.sp.shift[c] + m;
    if (std_out) std_out[o] = sd;
}

template <typename TOut>
__device__ __forceinline__ void store_out(TOut *p, double v) { *p = (TOut)v; }

// Thread per (fold p, upper-triangle element (i, j) of one H tile) with i < K
// and i <= j < K + M:
//   G'_T = G'_R - G'_p                                (Lemmas 2, 3)
//   centered:   v = G'_T - S'_T,i S'_T,j / N_T        (Propositions 7, 8;
//               X^T Y is centered when X or Y is, Lemma 9 / Table 1)
//   uncentered: v = G'_T + s_i S'_T,j + S'_T,i s_j + N_T s_i s_j
//               (expanding (x' + s_i)(z' + s_j) over T)
//   scaled:     v /= sigma_i sigma_j                   (Propositions 15, 16)
// X^T X entries are written to (i, j) and (j, i) from the same value.
template <typename TOut>
__global__ void __launch_bounds__(256) k_epilogue(PlanView pl, int flags, TOut *__restrict__ XTX,
                                                  TOut *__restrict__ XTY) {
    const int tile = blockIdx.y;
    const int p = blockIdx.z;
    const TileCoord tc = pl.tiles[tile];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = tc.bi * TILE + e % TILE;   // column-major partial tiles
    const int j = tc.bj * TILE + e / TILE;
    const int K = pl.K, M = pl.M, KM = K + M;
    if (i >= K || j < i || j >= KM) return;
    const bool is_xx = j < K;
    if (is_xx ? XTX == nullptr : XTY == nullptr) return;
    const bool cx = flags & CV_CENTER_X, sx = flags & CV_SCALE_X;
    const bool cy = flags & CV_CENTER_Y, sy = flags & CV_SCALE_Y;
    const bool centered = is_xx ? cx : (cx || cy);
    const bool scale_i = sx, scale_j = is_xx ? sx : sy;
    const double isc = pl.sp.inv_scale[i] * pl.sp.inv_scale[j];
    const double nt = (double)(pl.N - (pl.offs[p + 1] - pl.offs[p]));
    const double gt = (pl.gtot[(int64_t)tile * TILE_ELEMS + e] - gfold_at(pl, p, tile, e)) * isc;
    const double sti = pl.stats[2 * ((int64_t)p * KM + i)];
    const double stj = pl.stats[2 * ((int64_t)p * KM + j)];
    double v;
    if (centered) {
        v = gt - sti * (stj / nt);
    } else {
        const double si = pl.sp.shift[i], sj = pl.sp.shift[j];
        v = gt + si * stj + sti * sj + nt * si * sj;
    }
    const double di = scale_i ? pl.stats[2 * ((int64_t)p * KM + i) + 1] : 1.0;
    const double dj = scale_j ? pl.stats[2 * ((int64_t)p * KM + j) + 1] : 1.0;
    if (scale_i || scale_j) v = v / (di * dj);
    if (is_xx) {
        TOut *o = XTX + (int64_t)p * K * K;
        store_out(o + (int64_t)i * K + j, v);
        if (i != j) store_out(o + (int64_t)j * K + i, v);
    } else {
        store_out(XTY + (int64_t)p * K * M + (int64_t)i * M + (j - K), v);
    }
}

}  // namespace

cudaError_t shift_estimate(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y,
                           int64_t ldy, bool split, cudaStream_t st) {
    const PlanView &v = pl->v;
    const int S = (int)(v.N < SHIFT_SAMPLE ? v.N : SHIFT_SAMPLE);
    const int blocks = (v.D + 31) / 32;
    if (pl->in_dtype == CV_F32)
        k_shift_estimate<float><<<blocks, SHIFT_WARPS * 32, 0, st>>>((const float *)X, ldx, (const float *)Y, ldy,
                                                        v.N, v.K, v.M, S, split, v.int_bits, v.sp);
    else
        k_shift_estimate<double><<<blocks, SHIFT_WARPS * 32, 0, st>>>((const double *)X, ldx, (const double *)Y,
                                                         ldy, v.N, v.K, v.M, S, split, v.int_bits, v.sp);
    return cudaGetLastError();
}

cudaError_t fold_stats(const cv_plan_s *pl, int ddof, double *mean_out, double *std_out,
                       cudaStream_t st) {
    const int KM = pl->v.K + pl->v.M;
    k_fold_reduce<<<dim3(TILE_ELEMS / 256, pl->v.ntiles), 256, 0, st>>>(pl->v);
    k_fold_stats<<<dim3((KM + 127) / 128, pl->v.P), 128, 0, st>>>(pl->v, ddof, mean_out, std_out);
    return cudaGetLastError();
}

cudaError_t epilogue(const cv_plan_s *pl, int flags, void *XTX, void *XTY, cudaStream_t st) {
    dim3 grid(TILE_ELEMS / 256, pl->v.ntiles, pl->v.P);
    if (pl->out_dtype == CV_F64)
        k_epilogue<double><<<grid, 256, 0, st>>>(pl->v, flags, (double *)XTX, (double *)XTY);
    else
        k_epilogue<float><<<grid, 256, 0, st>>>(pl->v, flags, (float *)XTX, (float *)XTY);
    return cudaGetLastError();
}

}  // namespace cvx
