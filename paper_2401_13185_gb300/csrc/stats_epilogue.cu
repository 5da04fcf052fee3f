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

constexpr int SHIFT_SAMPLE = 4096;

template <typename T>
__device__ __forceinline__ double load_w(const T *X, int64_t ldx, const T *Y, int64_t ldy, int K,
                                         int M, int64_t n, int c) {
    if (c < K) return (double)X[n * ldx + c];
    if (c < K + M) return (double)Y[n * ldy + (c - K)];
    return 1.0;
}

// One block per 32 columns; lane = column, warp w takes sample rows w, w+8, ...
template <typename T>
__global__ void k_shift_estimate(const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y,
                                 int64_t ldy, int64_t N, int K, int M, int S, bool split,
                                 ShiftParams sp) {
    __shared__ double red[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const int D = K + M + 1;
    const bool live = c < K + M;
    double sum = 0.0;
    if (live)
        for (int k = warp; k < S; k += 8) sum += load_w(X, ldx, Y, ldy, K, M, (k * N) / S, c);
    red[warp][lane] = sum;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][lane];
    s /= (double)S;
    if (sizeof(T) == 4) s = (double)(float)s;   // FP32 inputs: x - s exact in FP64
    __syncthreads();
    double mx = 0.0;
    if (live && split)
        for (int k = warp; k < S; k += 8)
            mx = fmax(mx, fabs(load_w(X, ldx, Y, ldy, K, M, (k * N) / S, c) - s));
    red[warp][lane] = mx;
    __syncthreads();
    if (warp == 0 && c < D) {
        double m = 0.0;
        for (int w = 0; w < 8; ++w) m = fmax(m, red[w][lane]);
        int e = 0;
        if (!live) {
            s = 0.0;   // the ones column
        } else if (split && m > 0.0) {
            int ex;
            frexp(m, &ex);          // m < 2^ex
            e = 8 - ex;             // m * 2^e < 2^8, leaving 2^8 headroom below FP16's max
            e = max(-120, min(120, e));
        }
        sp.shift[c] = s;
        sp.shift_f[c] = (float)s;
        sp.scale_f[c] = ldexpf(1.0f, e);
        sp.inv_scale[c] = ldexp(1.0, -e);
    }
}

__device__ __forceinline__ const double *partial_tile(const PlanView &pl, int seg, int tile) {
    return pl.partials + ((int64_t)seg * pl.ntiles + tile) * TILE_ELEMS;
}

// Thread per column c < K + M.  stats[(p * (K+M) + c) * 2] = {S'_T, sigma}.
__global__ void k_fold_stats(PlanView pl, int ddof, double *__restrict__ mean_out,
                             double *__restrict__ std_out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int KM = pl.K + pl.M;
    if (c >= KM) return;
    const int ones = pl.D - 1;
    const int t_sum = tile_index(pl.nb, c / TILE, ones / TILE);
    const int e_sum = (c % TILE) * TILE + (ones % TILE);
    const int t_sq = tile_index(pl.nb, c / TILE, c / TILE);
    const int e_sq = (c % TILE) * TILE + (c % TILE);
    const double isc = pl.sp.inv_scale[c];
    double s_all = 0.0, q_all = 0.0;
    for (int g = 0; g < pl.nsegs; ++g) {
        s_all += partial_tile(pl, g, t_sum)[e_sum];
        q_all += partial_tile(pl, g, t_sq)[e_sq];
    }
    const double shift = pl.sp.shift[c];
    for (int p = 0; p < pl.P; ++p) {
        double s_v = 0.0, q_v = 0.0;
        for (int g = pl.fold_seg[p]; g < pl.fold_seg[p + 1]; ++g) {
            s_v += partial_tile(pl, g, t_sum)[e_sum];
            q_v += partial_tile(pl, g, t_sq)[e_sq];
        }
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
        if (mean_out) mean_out[o] = shift + m;
        if (std_out) std_out[o] = sd;
    }
}

template <typename TOut>
__device__ __forceinline__ void store_out(TOut *p, double v) { *p = (TOut)v; }

// Thread per upper-triangle element (i, j) of one H tile with i < K and
// i <= j < K + M.  For every fold p:
//   G'_T = G'_R - G'_p                                (Lemma 2 / 3)
//   centered:   v = G'_T - S'_T,i S'_T,j / N_T        (Propositions 7, 8;
//               X^T Y is centered when X or Y is, Lemma 9 / Table 1)
//   uncentered: v = G'_T + s_i S'_T,j + S'_T,i s_j + N_T s_i s_j
//               (expanding (x' + s_i)(z' + s_j) over T)
//   scaled:     v /= sigma_i sigma_j                   (Propositions 15, 16)
// X^T X entries are written to (i, j) and (j, i) from the same value.
template <typename TOut>
__global__ void k_epilogue(PlanView pl, int flags, TOut *__restrict__ XTX, TOut *__restrict__ XTY) {
    const int tile = blockIdx.y;
    const TileCoord tc = pl.tiles[tile];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= TILE_ELEMS) return;
    const int i = tc.bi * TILE + e / TILE;
    const int j = tc.bj * TILE + e % TILE;
    const int K = pl.K, M = pl.M, KM = K + M;
    if (i >= K || j < i || j >= KM) return;
    const bool is_xx = j < K;
    if (is_xx ? XTX == nullptr : XTY == nullptr) return;
    const bool cx = flags & CV_CENTER_X, sx = flags & CV_SCALE_X;
    const bool cy = flags & CV_CENTER_Y, sy = flags & CV_SCALE_Y;
    const bool centered = is_xx ? cx : (cx || cy);
    const bool scale_i = sx, scale_j = is_xx ? sx : sy;
    const double isc = pl.sp.inv_scale[i] * pl.sp.inv_scale[j];
    const double si = pl.sp.shift[i], sj = pl.sp.shift[j];
    double g_all = 0.0;
    for (int g = 0; g < pl.nsegs; ++g) g_all += partial_tile(pl, g, tile)[e];
    for (int p = 0; p < pl.P; ++p) {
        double g_v = 0.0;
        for (int g = pl.fold_seg[p]; g < pl.fold_seg[p + 1]; ++g) g_v += partial_tile(pl, g, tile)[e];
        const double nt = (double)(pl.N - (pl.offs[p + 1] - pl.offs[p]));
        const double gt = (g_all - g_v) * isc;
        const double sti = pl.stats[2 * ((int64_t)p * KM + i)];
        const double stj = pl.stats[2 * ((int64_t)p * KM + j)];
        double v;
        if (centered) v = gt - sti * (stj / nt);
        else v = gt + si * stj + sti * sj + nt * si * sj;
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
}

}  // namespace

cudaError_t shift_estimate(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y,
                           int64_t ldy, bool split, cudaStream_t st) {
    const PlanView &v = pl->v;
    const int S = (int)(v.N < SHIFT_SAMPLE ? v.N : SHIFT_SAMPLE);
    const int blocks = (v.D + 31) / 32;
    if (pl->in_dtype == CV_F32)
        k_shift_estimate<float><<<blocks, 256, 0, st>>>((const float *)X, ldx, (const float *)Y, ldy,
                                                        v.N, v.K, v.M, S, split, v.sp);
    else
        k_shift_estimate<double><<<blocks, 256, 0, st>>>((const double *)X, ldx, (const double *)Y,
                                                         ldy, v.N, v.K, v.M, S, split, v.sp);
    return cudaGetLastError();
}

cudaError_t fold_stats(const cv_plan_s *pl, int ddof, double *mean_out, double *std_out,
                       cudaStream_t st) {
    const int KM = pl->v.K + pl->v.M;
    k_fold_stats<<<(KM + 127) / 128, 128, 0, st>>>(pl->v, ddof, mean_out, std_out);
    return cudaGetLastError();
}

cudaError_t epilogue(const cv_plan_s *pl, int flags, void *XTX, void *XTY, cudaStream_t st) {
    dim3 grid(TILE_ELEMS / 256, pl->v.ntiles);
    if (pl->out_dtype == CV_F64)
        k_epilogue<double><<<grid, 256, 0, st>>>(pl->v, flags, (double *)XTX, (double *)XTY);
    else
        k_epilogue<float><<<grid, 256, 0, st>>>(pl->v, flags, (float *)XTX, (float *)XTY);
    return cudaGetLastError();
}

}  // namespace cvx
