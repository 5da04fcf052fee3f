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

#include <algorithm>

#include "cvx_internal.cuh"

namespace cvx {
namespace {

constexpr int MAX_GRID_FOLDS = 65535;   // grid y / z limit

// Shift estimate over a strided sample of S <= SHIFT_SAMPLE rows (row
// indices k N / S, precomputed by the plan), in two kernels so that the
// sample's loads spread over many SMs:
//   k_shift_partial  block (32 columns, chunk of SHIFT_ROWS_PER_CHUNK sample
//                    rows): per column, the sum, minimum and maximum of the
//                    deviations x - v0 from the column's first sampled value,
//                    in FP32 (the shift is only an estimate, any value keeps
//                    the results exact; FP64 is slow on this part);
//   k_shift_final    thread per column: combines the chunks in a fixed order,
//                    s = v0 + mean deviation (so a constant column gets its
//                    constant exactly), and the power-of-two scale from the
//                    largest deviation from s.
template <typename T>
__device__ __forceinline__ void column_ptr(const T *X, int64_t ldx, const T *Y, int64_t ldy, int K, int M, int c,
                                           const T *&col, int64_t &ld) {
    const bool live = c < K + M;
    col = !live ? X : (c < K ? X + c : Y + (c - K));
    ld = !live ? 0 : (c < K ? ldx : ldy);
}

template <typename T>
__global__ void __launch_bounds__(128) k_shift_partial(const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y,
                                                        int64_t ldy, const int32_t *__restrict__ rows, int K, int M,
                                                        int S, float *__restrict__ part) {
    __shared__ float red[3][4][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const int D = K + M + 1;
    const T *col;
    int64_t ld;
    column_ptr(X, ldx, Y, ldy, K, M, c, col, ld);
    const T v0 = col[(int64_t)rows[0] * ld];
    constexpr int PER = SHIFT_ROWS_PER_CHUNK / 4;
    float dev[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int k = blockIdx.y * SHIFT_ROWS_PER_CHUNK + warp * PER + j;
        dev[j] = k < S ? (float)(__ldg(col + (int64_t)rows[k] * ld) - v0) : 0.0f;
    }
    float sum = 0.0f, mn = 0.0f, mx = 0.0f;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int k = blockIdx.y * SHIFT_ROWS_PER_CHUNK + warp * PER + j;
        if (k < S) {
            sum += dev[j];
            mn = fminf(mn, dev[j]);
            mx = fmaxf(mx, dev[j]);
        }
    }
    red[0][warp][lane] = sum;
    red[1][warp][lane] = mn;
    red[2][warp][lane] = mx;
    __syncthreads();
    if (warp == 0 && c < D) {
        float a = 0.0f, b = 0.0f, d = 0.0f;
        for (int w = 0; w < 4; ++w) {
            a += red[0][w][lane];
            b = fminf(b, red[1][w][lane]);
            d = fmaxf(d, red[2][w][lane]);
        }
        float *o = part + ((int64_t)blockIdx.y * D + c) * 3;
        o[0] = a;
        o[1] = b;
        o[2] = d;
    }
}

template <typename T>
__global__ void k_shift_final(const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y, int64_t ldy,
                              const int32_t *__restrict__ rows, int K, int M, int S, int chunks, bool split,
                              int int_bits, const float *__restrict__ part, ShiftParams sp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int D = K + M + 1;
    if (c >= D) return;
    if (c >= K + M) {   // the ones column
        sp.shift[c] = 0.0;
        sp.shift_f[c] = 0.0f;
        sp.scale_f[c] = 1.0f;
        sp.inv_scale[c] = 1.0;
        return;
    }
    const T *col;
    int64_t ld;
    column_ptr(X, ldx, Y, ldy, K, M, c, col, ld);
    const T v0 = col[(int64_t)rows[0] * ld];
    float sum = 0.0f, mn = 0.0f, mx = 0.0f;
    for (int q = 0; q < chunks; ++q) {
        const float *o = part + ((int64_t)q * D + c) * 3;
        sum += o[0];
        mn = fminf(mn, o[1]);
        mx = fmaxf(mx, o[2]);
    }
    double s = (double)v0 + (double)(sum / (float)S);
    if (sizeof(T) == 4) s = (double)(float)s;   // FP32 inputs: x - s exact in FP64
    const double sd = s - (double)v0;
    const double m = fmax((double)mx - sd, sd - (double)mn);   // largest |x - s| in the sample
    int e = 0;
    if (split && m > 0.0) {
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

// Per-fold validation sums of H: thread per (fold p, tile, element); the
// fold's few segment partials are independent loads.  Split-path partials are
// summed exactly in int64 (hi * hi part) and in FP32 (cross terms, about 2^-B
// of the total): no FP64 arithmetic, which is slow on this part.
__global__ void __launch_bounds__(256) k_fold_sum(PlanView pl, int p_base) {
    const int tile = blockIdx.y, p = p_base + (int)blockIdx.z;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t seg_stride = (int64_t)pl.ntiles * TILE_ELEMS;
    const int64_t off = (int64_t)tile * TILE_ELEMS + e;
    const int64_t out = (int64_t)p * seg_stride + off;
    const int g0 = pl.fold_seg[p], g1 = pl.fold_seg[p + 1];
    if (pl.split) {
        const int32_t *__restrict__ hi = part_hi(pl) + off;
        const float *__restrict__ lo = part_lo(pl) + off;
        long long a0 = 0;
        float a1 = 0.0f;
        int g = g0;
        for (; g + 4 <= g1; g += 4) {
            const int32_t h0 = hi[(int64_t)g * seg_stride], h1 = hi[(int64_t)(g + 1) * seg_stride];
            const int32_t h2 = hi[(int64_t)(g + 2) * seg_stride], h3 = hi[(int64_t)(g + 3) * seg_stride];
            const float l0 = lo[(int64_t)g * seg_stride], l1 = lo[(int64_t)(g + 1) * seg_stride];
            const float l2 = lo[(int64_t)(g + 2) * seg_stride], l3 = lo[(int64_t)(g + 3) * seg_stride];
            a0 += (long long)h0 + h1 + h2 + h3;
            a1 += l0;
            a1 += l1;
            a1 += l2;
            a1 += l3;
        }
        for (; g < g1; ++g) {
            a0 += hi[(int64_t)g * seg_stride];
            a1 += lo[(int64_t)g * seg_stride];
        }
        long long *fold_hi = reinterpret_cast<long long *>(pl.gfold);
        float *fold_lo = reinterpret_cast<float *>(fold_hi + (int64_t)pl.P * seg_stride);
        fold_hi[out] = a0;
        fold_lo[out] = a1;
    } else {
        const double *__restrict__ src = pl.partials + off;
        double acc = 0.0;
        int g = g0;
        for (; g + 4 <= g1; g += 4) {
            const double a = src[(int64_t)g * seg_stride], b = src[(int64_t)(g + 1) * seg_stride];
            const double c = src[(int64_t)(g + 2) * seg_stride], d = src[(int64_t)(g + 3) * seg_stride];
            acc += a;
            acc += b;
            acc += c;
            acc += d;
        }
        for (; g < g1; ++g) acc += src[(int64_t)g * seg_stride];
        reinterpret_cast<double *>(pl.gfold)[out] = acc;
    }
}

// H over all rows: the fold sums added in fold order, 8 independent loads at
// a time (int64 + FP32 on the split path, FP64 otherwise).
__global__ void __launch_bounds__(256) k_total_sum(PlanView pl) {
    const int tile = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)pl.ntiles * TILE_ELEMS;
    const int64_t off = (int64_t)tile * TILE_ELEMS + e;
    constexpr int U = 8;
    if (pl.split) {
        const long long *fold_hi = reinterpret_cast<const long long *>(pl.gfold);
        const float *fold_lo = reinterpret_cast<const float *>(fold_hi + (int64_t)pl.P * nt);
        long long a0 = 0;
        float a1 = 0.0f;
        for (int p0 = 0; p0 < pl.P; p0 += U) {
            long long h[U];
            float l[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                h[u] = p0 + u < pl.P ? fold_hi[(int64_t)(p0 + u) * nt + off] : 0;
                l[u] = p0 + u < pl.P ? fold_lo[(int64_t)(p0 + u) * nt + off] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                a0 += h[u];
                a1 += l[u];
            }
        }
        long long *tot_hi = reinterpret_cast<long long *>(pl.gtot);
        float *tot_lo = reinterpret_cast<float *>(tot_hi + nt);
        tot_hi[off] = a0;
        tot_lo[off] = a1;
    } else {
        const double *src = reinterpret_cast<const double *>(pl.gfold) + off;
        double tot = 0.0;
        for (int p0 = 0; p0 < pl.P; p0 += U) {
            double v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = p0 + u < pl.P ? src[(int64_t)(p0 + u) * nt] : 0.0;
#pragma unroll
            for (int u = 0; u < U; ++u) tot += v[u];
        }
        reinterpret_cast<double *>(pl.gtot)[off] = tot;
    }
}

// Thread per (fold p, column c < K + M).  From the fold and total sums:
//   S'_T = S'_R - S'_p,  Q'_T = Q'_R - Q'_p        (Lemma 14, shifted units)
//   m'_T = S'_T / N_T                               (Lemma 7, written with sums)
//   var  = max(0, Q'_T - S'_T m'_T) / (N_T - ddof)  (Lemma 12 after substituting
//                                                   the mean; rounding below 0
//                                                   is clamped)
//   sigma = sqrt(var), replaced by 1 when var is 0  (Algorithm 7 step 24)
// and, with rho = 1 / sigma for a scaled side and 1 otherwise, the per-column
// factors of the epilogue:
//   A = 2^-e rho  (undoes the split path's power-of-two scale)
//   B = S'_T rho,  C = m'_T rho,  E = s rho  (s = the column's shift).
// The product entry (i, j) is then
//   centered    G A_i A_j - B_i C_j
//   uncentered  G A_i A_j + E_i B_j + B_i E_j + N_T E_i E_j
// with G the scaled training Gram entry, so the epilogue needs no division
// (FP64 division is costly on this part).
__global__ void k_fold_stats(PlanView pl, int flags, int ddof, double *__restrict__ mean_out,
                             double *__restrict__ std_out, int p_base) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = p_base + (int)blockIdx.y;
    const int KM = pl.K + pl.M;
    if (c >= KM) return;
    const int ones = pl.D - 1;
    const int t_sum = tile_index(pl.nb, c / TILE, ones / TILE);
    const int e_sum = (ones % TILE) * TILE + (c % TILE);   // column-major tiles
    const int t_sq = tile_index(pl.nb, c / TILE, c / TILE);
    const int e_sq = (c % TILE) * TILE + (c % TILE);
    const double isc = pl.sp.inv_scale[c];
    const double nt = (double)(pl.N - (pl.offs[p + 1] - pl.offs[p]));
    const double st = g_train(pl, p, t_sum, e_sum) * isc;
    const double qt = g_train(pl, p, t_sq, e_sq) * isc * isc;
    const double m = st / nt;
    double var = nt - ddof > 0 ? (qt - st * m) / (nt - ddof) : NAN;
    if (var < 0.0) var = 0.0;
    double sd = sqrt(var);
    if (var == 0.0) sd = 1.0;
    const bool scaled = c < pl.K ? (flags & CV_SCALE_X) : (flags & CV_SCALE_Y);
    const double rho = scaled ? 1.0 / sd : 1.0;
    const int64_t o = (int64_t)p * KM + c;
    pl.stats[4 * o + 0] = isc * rho;
    pl.stats[4 * o + 1] = st * rho;
    pl.stats[4 * o + 2] = m * rho;
    pl.stats[4 * o + 3] = pl.sp.shift[c] * rho;
    if (mean_out) mean_out[o] = pl.sp.shift[c] + m;
    if (std_out) std_out[o] = sd;
}

template <typename TOut>
__device__ __forceinline__ void store_out(TOut *p, double v) { *p = (TOut)v; }

// Value of output entry (i, j) of fold p (i < K, i <= j < K + M):
//   G'_T = G'_R - G'_p                                (Lemmas 2, 3)
//   centered:   v = G'_T - S'_T,i S'_T,j / N_T        (Propositions 7, 8;
//               X^T Y is centered when X or Y is, Lemma 9 / Table 1)
//   uncentered: v = G'_T + s_i S'_T,j + S'_T,i s_j + N_T s_i s_j
//               (expanding (x' + s_i)(z' + s_j) over T)
//   scaled:     v /= sigma_i sigma_j                   (Propositions 15, 16)
// evaluated with the per-column factors of k_fold_stats.
__device__ __forceinline__ double entry_value(const PlanView &pl, bool centered, int p, int tile, int e, int i,
                                              int j) {
    const int KM = pl.K + pl.M;
    const double g = g_train(pl, p, tile, e);
    const double *fi = pl.stats + 4 * ((int64_t)p * KM + i);
    const double *fj = pl.stats + 4 * ((int64_t)p * KM + j);
    const double aa = fi[0] * fj[0];
    if (centered) return fma(g, aa, -fi[1] * fj[2]);
    const double nt = (double)(pl.N - (pl.offs[p + 1] - pl.offs[p]));
    return fma(g, aa, fma(fi[3], fj[1], fma(fi[1], fj[3], nt * fi[3] * fj[3])));
}

// Block (32 x 8 threads) per (fold p, 32 x 32 sub-tile of one H tile).  Pass 1
// (thread x = row offset): writes X^T X (j, i) and X^T Y (i, j) with
// consecutive threads on consecutive i, and keeps the values in shared memory;
// pass 2 (thread x = column offset) writes X^T X (i, j), i < j, from the same
// values, so both triangles are written coalesced and bitwise symmetric.
template <typename TOut>
__global__ void __launch_bounds__(256) k_epilogue(PlanView pl, int flags, TOut *__restrict__ XTX,
                                                  TOut *__restrict__ XTY, int p_base) {
    __shared__ double vals[32][33];
    const int tile = blockIdx.y, p = p_base + (int)blockIdx.z;
    const TileCoord tc = pl.tiles[tile];
    const int si = blockIdx.x / 4, sj = blockIdx.x % 4;
    const int li0 = si * 32, lj0 = sj * 32;   // offsets inside the 128 x 128 tile
    const int i0 = tc.bi * TILE + li0, j0 = tc.bj * TILE + lj0;
    const int K = pl.K, M = pl.M, KM = K + M;
    if (i0 >= K || j0 >= KM || j0 + 31 < i0) return;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool cx = flags & CV_CENTER_X, cy = flags & CV_CENTER_Y;
    TOut *xtx = XTX ? XTX + (int64_t)p * K * K : nullptr;
    TOut *xty = XTY ? XTY + (int64_t)p * K * M : nullptr;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int li = tx, lj = ty + 8 * r;
        const int i = i0 + li, j = j0 + lj;
        const bool ok = i < K && j < KM && i <= j;
        double v = 0.0;
        if (ok) {
            const int e = (lj0 + lj) * TILE + (li0 + li);   // column-major tiles
            v = entry_value(pl, j < K ? cx : (cx || cy), p, tile, e, i, j);
            if (j < K) {
                if (xtx) xtx[(int64_t)j * K + i] = (TOut)v;
            } else if (xty) {
                xty[(int64_t)i * M + (j - K)] = (TOut)v;
            }
        }
        vals[lj][li] = v;
    }
    __syncthreads();
    if (!xtx) return;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int lj = tx, li = ty + 8 * r;
        const int i = i0 + li, j = j0 + lj;
        if (i < K && j < K && i < j) xtx[(int64_t)i * K + j] = (TOut)vals[lj][li];
    }
}

}  // namespace

cudaError_t shift_estimate(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y,
                           int64_t ldy, bool split, cudaStream_t st) {
    const PlanView &v = pl->v;
    const int S = v.nsample;
    const int chunks = (S + SHIFT_ROWS_PER_CHUNK - 1) / SHIFT_ROWS_PER_CHUNK;
    dim3 grid((v.D + 31) / 32, chunks);
    const int fb = (v.D + 127) / 128;
    if (pl->in_dtype == CV_F32) {
        k_shift_partial<float><<<grid, 128, 0, st>>>((const float *)X, ldx, (const float *)Y, ldy, v.sample_rows,
                                                     v.K, v.M, S, v.shift_part);
        k_shift_final<float><<<fb, 128, 0, st>>>((const float *)X, ldx, (const float *)Y, ldy, v.sample_rows, v.K,
                                                 v.M, S, chunks, split, v.int_bits, v.shift_part, v.sp);
    } else {
        k_shift_partial<double><<<grid, 128, 0, st>>>((const double *)X, ldx, (const double *)Y, ldy,
                                                      v.sample_rows, v.K, v.M, S, v.shift_part);
        k_shift_final<double><<<fb, 128, 0, st>>>((const double *)X, ldx, (const double *)Y, ldy, v.sample_rows,
                                                  v.K, v.M, S, chunks, split, v.int_bits, v.shift_part, v.sp);
    }
    return cudaGetLastError();
}

cudaError_t fold_stats(const cv_plan_s *pl, int flags, int ddof, double *mean_out, double *std_out,
                       cudaStream_t st) {
    const int KM = pl->v.K + pl->v.M;
    for (int p0 = 0; p0 < pl->v.P; p0 += MAX_GRID_FOLDS) {
        const int np = std::min(MAX_GRID_FOLDS, pl->v.P - p0);
        k_fold_sum<<<dim3(TILE_ELEMS / 256, pl->v.ntiles, np), 256, 0, st>>>(pl->v, p0);
    }
    k_total_sum<<<dim3(TILE_ELEMS / 256, pl->v.ntiles), 256, 0, st>>>(pl->v);
    for (int p0 = 0; p0 < pl->v.P; p0 += MAX_GRID_FOLDS) {
        const int np = std::min(MAX_GRID_FOLDS, pl->v.P - p0);
        k_fold_stats<<<dim3((KM + 127) / 128, np), 128, 0, st>>>(pl->v, flags, ddof, mean_out, std_out, p0);
    }
    return cudaGetLastError();
}

cudaError_t epilogue(const cv_plan_s *pl, int flags, void *XTX, void *XTY, cudaStream_t st) {
    dim3 block(32, 8);
    for (int p0 = 0; p0 < pl->v.P; p0 += MAX_GRID_FOLDS) {
        const int np = std::min(MAX_GRID_FOLDS, pl->v.P - p0);
        dim3 grid((TILE / 32) * (TILE / 32), pl->v.ntiles, np);
        if (pl->out_dtype == CV_F64)
            k_epilogue<double><<<grid, block, 0, st>>>(pl->v, flags, (double *)XTX, (double *)XTY, p0);
        else
            k_epilogue<float><<<grid, block, 0, st>>>(pl->v, flags, (float *)XTX, (float *)XTY, p0);
    }
    return cudaGetLastError();
}

}  // namespace cvx
