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
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>

#include "cvx_internal.cuh"

namespace cg = cooperative_groups;

namespace cvx {
namespace {

constexpr int MAX_GRID_FOLDS = 65535;   // grid y / z limit

// Shift estimate over a strided sample of S <= SHIFT_SAMPLE rows (row k of
// the sample is row k N / S).  A cluster of SHIFT_CHUNKS blocks serves a
// group of 32 columns; block q of the cluster takes sample rows
// q SHIFT_ROWS_PER_CHUNK .. + SHIFT_ROWS_PER_CHUNK - 1 and forms, per column,
// the sum, minimum and maximum of the deviations x - v0 from the column's
// value in row 0, in FP32 (the shift is only an estimate: any value keeps the
// results exact; FP64 is slow on this part).  After a cluster barrier, block
// 0 reads the other blocks' partials from their shared memory and combines
// them in block order: s = v0 + mean deviation (a constant column gets its
// constant exactly), and for the split path the power-of-two scale from the
// largest deviation from s.  A second cluster barrier keeps the partials
// alive until block 0 has read them.
//
// Extra clusters past the shift clusters pack Y for the split path's bulk
// copies (FP32 inputs): Yp[n][j] = Y[n][j] (j < M), 1 (j == M), 0 (M < j < mp),
// i.e. Y and the ones column of W in 16-byte aligned rows.
template <typename T>
__device__ __forceinline__ void column_ptr(const T *X, int64_t ldx, const T *Y, int64_t ldy, int K, int M, int c,
                                           const T *&col, int64_t &ld) {
    const bool live = c < K + M;
    col = !live ? X : (c < K ? X + c : Y + (c - K));
    ld = !live ? 0 : (c < K ? ldx : ldy);
}

constexpr int SHIFT_CHUNKS = SHIFT_SAMPLE / SHIFT_ROWS_PER_CHUNK;   // blocks per cluster

struct ShiftArgs {
    int64_t N;
    int K, M, S, groups;
    int split, int_bits;
    ShiftParams sp;
    float *ypack;     // N x mp, or null: no packing clusters
    int mp;
};

template <typename T>
__device__ __forceinline__ void shift_cluster(const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y, int64_t ldy,
                                              const ShiftArgs &a, int g);

template <typename T>
__global__ void __cluster_dims__(SHIFT_CHUNKS, 1, 1) __launch_bounds__(128)
    k_shift(const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y, int64_t ldy, ShiftArgs a) {
    grid_dep_wait();
    grid_dep_launch();
    const int tid = threadIdx.x;
    const int g = (int)blockIdx.x / SHIFT_CHUNKS;   // cluster: column group, or packing
    if (g >= a.groups) {
        // packing: thread per row, the row's M values then 1 and zeros, as
        // 16-byte stores (mp is a multiple of 4)
        if constexpr (sizeof(T) == 4) {
            const int nshift = a.groups * SHIFT_CHUNKS;
            const int64_t stride = (int64_t)(gridDim.x - nshift) * blockDim.x;
            for (int64_t n = (int64_t)(blockIdx.x - nshift) * blockDim.x + tid; n < a.N; n += stride) {
                const T *yr = Y + n * ldy;
                float4 *out = reinterpret_cast<float4 *>(a.ypack + n * a.mp);
                for (int j0 = 0; j0 < a.mp; j0 += 4) {
                    float w[4];
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const int j = j0 + d;
                        w[d] = j < a.M ? (float)yr[j] : (j == a.M ? 1.0f : 0.0f);
                    }
                    out[j0 / 4] = make_float4(w[0], w[1], w[2], w[3]);
                }
            }
        }
        return;
    }
    shift_cluster<T>(X, ldx, Y, ldy, a, g);
}

// Batched: cluster c takes (problem, column group) shift_units[c] of the batch.
__global__ void __cluster_dims__(SHIFT_CHUNKS, 1, 1) __launch_bounds__(128)
    k_shift_batched(const __grid_constant__ BatchTables bt, const __grid_constant__ BatchArgs ba) {
    grid_dep_wait();
    grid_dep_launch();
    const int2 u = bt.shift_units[blockIdx.x / SHIFT_CHUNKS];
    const PlanView &pl = bt.views[u.x];
    const ProblemArgs &pa = batch_arg(bt, ba, u.x);
    ShiftArgs a;
    a.N = pl.N;
    a.K = pl.K;
    a.M = pl.M;
    a.S = pl.nsample;
    a.groups = (pl.D + 31) / 32;
    a.split = pl.split;
    a.int_bits = pl.int_bits;
    a.sp = pl.sp;
    a.ypack = nullptr;
    a.mp = 0;
    shift_cluster<float>((const float *)pa.X, pa.ldx, (const float *)pa.Y, pa.ldy, a, u.y);
}

template <typename T>
__device__ __forceinline__ void shift_cluster(const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y, int64_t ldy,
                                              const ShiftArgs &a, int g) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    __shared__ float red[3][4][32];
    __shared__ float part[3][32];   // this block's per-column sum, minimum, maximum
    __shared__ int64_t rows[SHIFT_ROWS_PER_CHUNK];
    {   // this chunk's sample rows, one 64-bit division per thread
        const int k = q * SHIFT_ROWS_PER_CHUNK + tid;
        rows[tid] = k < a.S ? ((int64_t)k * a.N) / a.S : 0;
    }
    __syncthreads();
    const int c = g * 32 + lane;
    const int K = a.K, M = a.M, D = K + M + 1, S = a.S;
    const T *col;
    int64_t ld;
    column_ptr(X, ldx, Y, ldy, K, M, c, col, ld);
    const T v0 = col[0];
    constexpr int PER = SHIFT_ROWS_PER_CHUNK / 4;
    float dev[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int k = q * SHIFT_ROWS_PER_CHUNK + warp * PER + j;
        dev[j] = k < S ? (float)(__ldg(col + rows[warp * PER + j] * ld) - v0) : 0.0f;
    }
    float sum = 0.0f, mn = 0.0f, mx = 0.0f;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int k = q * SHIFT_ROWS_PER_CHUNK + warp * PER + j;
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
    if (warp == 0) {
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
        for (int w = 0; w < 4; ++w) {
            s0 += red[0][w][lane];
            s1 = fminf(s1, red[1][w][lane]);
            s2 = fmaxf(s2, red[2][w][lane]);
        }
        part[0][lane] = s0;
        part[1][lane] = s1;
        part[2][lane] = s2;
    }
    cluster.sync();
    if (q == 0 && warp == 0 && c < D) {
        if (c >= K + M) {   // the ones column
            a.sp.shift[c] = 0.0;
            a.sp.shift_f[c] = 0.0f;
            a.sp.scale_f[c] = 1.0f;
            a.sp.inv_scale[c] = 1.0;
        } else {
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
            for (int r = 0; r < SHIFT_CHUNKS; ++r) {
                const float *pr = cluster.map_shared_rank(&part[0][0], r);
                s0 += pr[lane];
                s1 = fminf(s1, pr[32 + lane]);
                s2 = fmaxf(s2, pr[64 + lane]);
            }
            double sh = (double)v0 + (double)(s0 / (float)S);
            if (sizeof(T) == 4) sh = (double)(float)sh;   // FP32 inputs: x - s exact in FP64
            const double sd = sh - (double)v0;
            const double m = fmax((double)s2 - sd, sd - (double)s1);   // largest |x - s| in the sample
            int e = 0;
            if (a.split && m > 0.0) {
                int ex;
                frexp(m, &ex);            // m < 2^ex
                e = a.int_bits - ex;      // sampled max * 2^e < 2^int_bits
                e = max(-120, min(120, e));
            }
            a.sp.shift[c] = sh;
            a.sp.shift_f[c] = (float)sh;
            a.sp.scale_f[c] = ldexpf(1.0f, e);
            a.sp.inv_scale[c] = ldexp(1.0, -e);
        }
    }
    cluster.sync();   // the partials stay in shared memory until block 0 has read them
}

// FP64 path: per-fold validation sums of H, thread per (fold p, tile,
// element); the fold's few segment partials are independent loads.  Fold p's
// sums go to dst + p * ntiles * TILE_ELEMS (the fold sums, or with the
// small-fold strategy's single pseudo-fold, the total).
__global__ void __launch_bounds__(256) k_fold_sum(PlanView pl, int p_base, double *__restrict__ dst) {
    grid_dep_wait();
    grid_dep_launch();
    const int tile = blockIdx.y, p = p_base + (int)blockIdx.z;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t seg_stride = (int64_t)pl.ntiles * TILE_ELEMS;
    const int64_t off = (int64_t)tile * TILE_ELEMS + e;
    const int64_t out = (int64_t)p * seg_stride + off;
    const int g0 = pl.fold_seg[p], g1 = pl.fold_seg[p + 1];
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
    dst[out] = acc;
}

// Split path: the total over the segment partials, thread per (tile, two
// consecutive elements), 8-byte loads.  The thread walks all segments in
// order, sixteen at a time with every load in flight at once; the hi * hi
// parts add exactly in int64 and the cross terms in FP32.  Each fold's sums
// (its segments in order, as fold_sum_split forms them) are added, in fold
// order, into the total (Lemma 2: H over all rows is the sum of the fold
// sums).  The small-fold strategy passes one pseudo-fold holding every
// segment.
__global__ void __launch_bounds__(256, 2) k_fold_total_split(PlanView pl, int nfold, long long *__restrict__ tot_hi,
                                                             float *__restrict__ tot_lo) {
    grid_dep_wait();
    grid_dep_launch();
    const int tile = blockIdx.y;
    const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int64_t seg_stride = (int64_t)pl.ntiles * TILE_ELEMS;
    const int64_t off = (int64_t)tile * TILE_ELEMS + e;
    const int32_t *__restrict__ hi = part_hi(pl) + off;
    const float *__restrict__ lo = part_lo(pl) + off;
    const int nseg = nfold > 0 ? pl.fold_seg[nfold] : pl.nsegs;
    long long fa0 = 0, fa1 = 0, ta0 = 0, ta1 = 0;
    float fb0 = 0.0f, fb1 = 0.0f, tb0 = 0.0f, tb1 = 0.0f;
    int p = 0;
    int p_end = nfold > 0 ? pl.fold_seg[1] : nseg;   // first segment past fold p
    constexpr int U = 16;
    for (int g0 = 0; g0 < nseg; g0 += U) {
        int2 h[U];
        float2 l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (g0 + u < nseg) {
                h[u] = __ldcs(reinterpret_cast<const int2 *>(hi + (int64_t)(g0 + u) * seg_stride));
                l[u] = __ldcs(reinterpret_cast<const float2 *>(lo + (int64_t)(g0 + u) * seg_stride));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = g0 + u;
            if (g < nseg) {
                while (g >= p_end) {   // leaving fold p
                    ta0 += fa0;
                    ta1 += fa1;
                    tb0 += fb0;
                    tb1 += fb1;
                    fa0 = fa1 = 0;
                    fb0 = fb1 = 0.0f;
                    ++p;
                    p_end = pl.fold_seg[p + 1];
                }
                fa0 += h[u].x;
                fa1 += h[u].y;
                fb0 += l[u].x;
                fb1 += l[u].y;
            }
        }
    }
    ta0 += fa0;
    ta1 += fa1;
    tb0 += fb0;
    tb1 += fb1;
    *reinterpret_cast<longlong2 *>(tot_hi + off) = make_longlong2(ta0, ta1);
    *reinterpret_cast<float2 *>(tot_lo + off) = make_float2(tb0, tb1);
}

// FP64 path: H over all rows, the fold sums added in fold order, 8
// independent loads at a time.
__global__ void __launch_bounds__(256) k_total_sum(PlanView pl) {
    grid_dep_wait();
    grid_dep_launch();
    const int tile = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)pl.ntiles * TILE_ELEMS;
    const int64_t off = (int64_t)tile * TILE_ELEMS + e;
    constexpr int U = 8;
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
//
// Split path: the factors are also stored in FP32 relative to a per-column
// power of two u = 2^t (t from the larger of |E| and A 2^int_bits, i.e. of
// the column's magnitude after preprocessing), so that the epilogue can form
// entry / (u_i u_j) in FP32 without overflow or underflow and attach
// 2^(t_i + t_j) exactly when it widens the result to FP64.
// Statistics and epilogue factors of fold p, column c, from the training sums
// in contraction units (S'_T and Q'_T before the power-of-two scale is undone).
// Per-fold constants of the statistics: 1 / N_T and 1 / (N_T - ddof) (NaN
// when N_T <= ddof), one division each per block instead of per thread (FP64
// division is slow on this part).
struct FoldRecip {
    double r_nt, r_dof;
};

__device__ __forceinline__ FoldRecip fold_recip(const PlanView &pl, int p, int ddof) {
    __shared__ FoldRecip fr;
    if (threadIdx.x == 0) {
        const double nt = (double)(pl.N - (pl.offs[p + 1] - pl.offs[p]));
        fr.r_nt = 1.0 / nt;
        fr.r_dof = nt - ddof > 0 ? 1.0 / (nt - ddof) : NAN;
    }
    __syncthreads();
    return fr;
}

__device__ __forceinline__ void finish_stats(const PlanView &pl, int flags, int ddof, int p, int c, double s_raw,
                                             double q_raw, FoldRecip fr, double *__restrict__ mean_out,
                                             double *__restrict__ std_out) {
    const int KM = pl.K + pl.M;
    const double isc = pl.sp.inv_scale[c];
    const double st = s_raw * isc, qt = q_raw * isc * isc;
    const double m = st * fr.r_nt;
    double var = (qt - st * m) * fr.r_dof;
    if (var < 0.0) var = 0.0;
    double sd = sqrt(var);
    if (var == 0.0) sd = 1.0;
    const bool scaled = c < pl.K ? (flags & CV_SCALE_X) : (flags & CV_SCALE_Y);
    const double rho = scaled ? 1.0 / sd : 1.0;
    const int64_t o = (int64_t)p * KM + c;
    const int64_t o_out = (int64_t)(p - pl.p_lo) * KM + c;   // outputs hold the plan's folds only
    const double A = isc * rho, B = st * rho, C = m * rho, E = pl.sp.shift[c] * rho;
    if (!pl.fac_f) {   // FP64 epilogue factors
        pl.stats[4 * o + 0] = A;
        pl.stats[4 * o + 1] = B;
        pl.stats[4 * o + 2] = C;
        pl.stats[4 * o + 3] = E;
    } else {
        // t = floor(log2 max(|E|, A 2^int_bits)); A, B, C, E then scaled by
        // the exact power of two 2^-t (A > 0 is normal: a power of two over sigma)
        const double big = fmax(fabs(E), A * pow2i(pl.int_bits));
        const int t = max(-1022, min(1022, ilogb_normal(big)));
        const double u = pow2i(-t);
        pl.fac_f[o] = make_float4((float)(A * u), (float)(B * u), (float)(C * u), (float)(E * u));
        pl.fac_t[o] = t;
    }
    if (mean_out) mean_out[o_out] = pl.sp.shift[c] + m;
    if (std_out) std_out[o_out] = sd;
}

// Tile index and column-major element of H holding (row c, column d).
__device__ __forceinline__ void h_element(const PlanView &pl, int c, int d, int &tile, int &e) {
    tile = tile_index(pl.nb, c / TILE, d / TILE);
    e = (d % TILE) * TILE + (c % TILE);
}

__global__ void k_fold_stats(PlanView pl, int flags, int ddof, double *__restrict__ mean_out,
                             double *__restrict__ std_out, int p_base) {
    grid_dep_wait();
    grid_dep_launch();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = p_base + (int)blockIdx.y;
    const int KM = pl.K + pl.M;
    const FoldRecip fr = fold_recip(pl, p, ddof);
    if (c >= KM) return;
    int t_sum, e_sum, t_sq, e_sq;
    h_element(pl, c, pl.D - 1, t_sum, e_sum);   // sum: the ones column
    h_element(pl, c, c, t_sq, e_sq);            // sum of squares: the diagonal
    double s_raw, q_raw;
    if (pl.small) {   // small-fold strategy: the fold's own sums come from its rows
        double sp, qp;
        if (pl.split) {
            const float2 f = reinterpret_cast<const float2 *>(pl.fold_sq)[(int64_t)p * KM + c];
            sp = f.x;
            qp = f.y;
        } else {
            const double2 f = reinterpret_cast<const double2 *>(pl.fold_sq)[(int64_t)p * KM + c];
            sp = f.x;
            qp = f.y;
        }
        s_raw = g_total(pl, t_sum, e_sum) - sp;
        q_raw = g_total(pl, t_sq, e_sq) - qp;
    } else {
        s_raw = g_train(pl, p, t_sum, e_sum);
        q_raw = g_train(pl, p, t_sq, e_sq);
    }
    finish_stats(pl, flags, ddof, p, c, s_raw, q_raw, fr, mean_out, std_out);
}

// Split path, fold-grouped strategy with at most FOLD_SMEM_MAX folds: the
// statistics straight from the segment partials, without the fold-sum pass.
// Thread per (column c, fold p) walks every segment's partial of the two
// elements (c, ones) and (c, c), 32 segments at a time, adding all of them
// into the totals and fold p's segments into the fold sums (exact int64 for
// hi * hi, FP32 for the cross terms, in segment order); the training sums are
// total - fold (Lemmas 2, 3, 14).
__device__ __forceinline__ void split_stats_body(const PlanView &pl, int flags, int ddof, double *__restrict__ mean_out,
                                                 double *__restrict__ std_out, int c, int p) {
    const FoldRecip fr = fold_recip(pl, p, ddof);
    if (c >= pl.K + pl.M) return;
    int t_sum, e_sum, t_sq, e_sq;
    h_element(pl, c, pl.D - 1, t_sum, e_sum);
    h_element(pl, c, c, t_sq, e_sq);
    const int64_t seg_stride = (int64_t)pl.ntiles * TILE_ELEMS;
    const int32_t *hs = part_hi(pl) + (int64_t)t_sum * TILE_ELEMS + e_sum;
    const int32_t *hq = part_hi(pl) + (int64_t)t_sq * TILE_ELEMS + e_sq;
    const float *ls = part_lo(pl) + (int64_t)t_sum * TILE_ELEMS + e_sum;
    const float *lq = part_lo(pl) + (int64_t)t_sq * TILE_ELEMS + e_sq;
    const int g0p = pl.fold_seg[p], g1p = pl.fold_seg[p + 1];
    long long ts = 0, tq = 0, fs = 0, fq = 0;
    float tsl = 0.0f, tql = 0.0f, fsl = 0.0f, fql = 0.0f;
    constexpr int U = 32;
    for (int g0 = 0; g0 < pl.nsegs; g0 += U) {
        int32_t a[U], b[U];
        float x[U], y[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (g0 + u < pl.nsegs) {
                const int64_t o = (int64_t)(g0 + u) * seg_stride;
                a[u] = __ldcg(hs + o);
                b[u] = __ldcg(hq + o);
                x[u] = __ldcg(ls + o);
                y[u] = __ldcg(lq + o);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = g0 + u;
            if (g < pl.nsegs) {
                ts += a[u];
                tq += b[u];
                tsl += x[u];
                tql += y[u];
                if (g >= g0p && g < g1p) {
                    fs += a[u];
                    fq += b[u];
                    fsl += x[u];
                    fql += y[u];
                }
            }
        }
    }
    finish_stats(pl, flags, ddof, p, c, (double)(ts - fs) + (double)(tsl - fsl), (double)(tq - fq) + (double)(tql - fql),
                 fr, mean_out, std_out);
}

__global__ void __launch_bounds__(32) k_split_stats(const __grid_constant__ PlanView pl, int flags, int ddof,
                                                    double *__restrict__ mean_out, double *__restrict__ std_out) {
    grid_dep_wait();
    grid_dep_launch();
    split_stats_body(pl, flags, ddof, mean_out, std_out, blockIdx.x * blockDim.x + threadIdx.x, (int)blockIdx.y);
}

// Batched: block per unit (problem, first column, fold) of the batch.
__global__ void __launch_bounds__(32) k_split_stats_batched(const __grid_constant__ BatchTables bt,
                                                            const __grid_constant__ BatchArgs ba) {
    grid_dep_wait();
    grid_dep_launch();
    const int4 u = bt.stats_units[blockIdx.x];
    const ProblemArgs &a = batch_arg(bt, ba, u.x);
    split_stats_body(bt.views[u.x], a.flags, a.ddof, a.mean_out, a.std_out, u.y + (int)threadIdx.x, u.z);
}

__device__ __forceinline__ double entry_value(const PlanView &pl, bool centered, int p, int tile, int e, int i,
                                              int j) {
    return entry_f64(pl, centered, p, i, j, g_train(pl, p, tile, e));
}

// Split path: G_T in FP32 from the exact int64 and FP32 sums, then entry_split.
__device__ __forceinline__ double entry_value_split(const PlanView &pl, bool centered, int p, int tile, int e,
                                                    int i, int j) {
    const int64_t nt = (int64_t)pl.ntiles * TILE_ELEMS;
    const int64_t it = (int64_t)tile * TILE_ELEMS + e;
    const long long *tot_hi = reinterpret_cast<const long long *>(pl.gtot);
    const float *tot_lo = reinterpret_cast<const float *>(tot_hi + nt);
    long long fh;
    float fl;
    fold_sum_split(pl, p, it, fh, fl);
    const float g = ll_to_float(tot_hi[it] - fh) + (tot_lo[it] - fl);
    return entry_split(pl, centered, p, i, j, g);
}

// Block (32 x 8 threads) per (fold p, 32 x 32 sub-tile of one H tile).  Pass 1
// (thread x = row offset): writes X^T X (j, i) and X^T Y (i, j) with
// consecutive threads on consecutive i, and keeps the values in shared memory;
// pass 2 (thread x = column offset) writes X^T X (i, j), i < j, from the same
// values, so both triangles are written coalesced and bitwise symmetric.
template <typename TOut, bool SPLIT>
__global__ void __launch_bounds__(256) k_epilogue(PlanView pl, int flags, TOut *__restrict__ XTX,
                                                  TOut *__restrict__ XTY, int p_base) {
    grid_dep_wait();
    grid_dep_launch();
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
    const int q = p - pl.p_lo;   // the fold's index in the outputs
    TOut *xtx = XTX ? XTX + (int64_t)q * xtx_fold_elems(pl) : nullptr;
    TOut *xty = XTY ? XTY + (int64_t)q * K * M : nullptr;
    const bool packed = pl.packed != 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int li = tx, lj = ty + 8 * r;
        const int i = i0 + li, j = j0 + lj;
        const bool ok = i < K && j < KM && i <= j;
        double v = 0.0;
        if (ok) {
            const int e = (lj0 + lj) * TILE + (li0 + li);   // column-major tiles
            const bool centered = j < K ? cx : (cx || cy);
            if constexpr (SPLIT)
                v = entry_value_split(pl, centered, p, tile, e, i, j);
            else
                v = entry_value(pl, centered, p, tile, e, i, j);
            if (j < K) {
                if (xtx && !packed) xtx[(int64_t)j * K + i] = (TOut)v;
            } else if (xty) {
                xty[(int64_t)i * M + (j - K)] = (TOut)v;
            }
        }
        vals[lj][li] = v;
    }
    __syncthreads();
    if (!xtx) return;
    // (i, j) above the diagonal from the transpose, consecutive threads on
    // consecutive j; the packed upper triangle takes the diagonal here too
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int lj = tx, li = ty + 8 * r;
        const int i = i0 + li, j = j0 + lj;
        if (i < K && j < K && (i < j || (packed && i == j)))
            xtx[packed ? packed_upper(K, i, j) : (int64_t)i * K + j] = (TOut)vals[lj][li];
    }
}

// Split path, fold-grouped strategy with at most FOLD_SMEM_MAX folds: the fold
// sums and the epilogue in one pass.  Block (16 x 16 threads) per (tile,
// 16 x 16 sub-tile); thread (x, y) owns H element (16 si + x, 16 sj + y) of the
// tile.  It walks every segment's partial of its element in order, sixteen
// segments' loads in flight at a time, keeps each fold's sum (exact int64 plus
// FP32) in shared memory and the total in registers, then for every fold forms
// G_T = total - fold (Lemmas 2, 3) and the entry (entry_split: Propositions 7,
// 8, 15, 16), and writes X^T X (j, i) and X^T Y (i, j) directly and X^T X
// (i, j) through a shared-memory transpose, so both triangles are written
// coalesced and bitwise symmetric.  Each partial is read once; no fold sums go
// through global memory.
constexpr int FOLD_SMEM_MAX = 32;

template <typename TOut>
__device__ __forceinline__ void fold_epilogue_body(const PlanView &pl, int flags, TOut *__restrict__ XTX,
                                                   TOut *__restrict__ XTY, int tile, int sub) {
    extern __shared__ uint8_t dyn[];
    long long *gh = reinterpret_cast<long long *>(dyn);                   // [P][256] fold sums, hi * hi
    float *gl = reinterpret_cast<float *>(gh + (int64_t)pl.P * 256);      // [P][256] cross terms
    float4 *fac = reinterpret_cast<float4 *>(gl + (int64_t)pl.P * 256);   // [P][32] factors of rows i, columns j
    int *fac_t = reinterpret_cast<int *>(fac + (int64_t)pl.P * 32);       // [P][32] their exponents
    float *ntr_s = reinterpret_cast<float *>(fac_t + (int64_t)pl.P * 32); // [P] N_T
    __shared__ double vals[2][16][17];
    const TileCoord tc = pl.tiles[tile];
    const int si = sub / 8, sj = sub % 8;
    const int li0 = 16 * si, lj0 = 16 * sj;
    const int i0 = tc.bi * TILE + li0, j0 = tc.bj * TILE + lj0;
    const int K = pl.K, M = pl.M, KM = K + M;
    if (i0 >= K || j0 >= KM || j0 + 15 < i0) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
    const int i = i0 + tx, j = j0 + ty;
    const bool ok = i < K && j < KM && i <= j;
    // every fold's factors of the block's 16 rows and 16 columns, loaded along
    // with the partials so that the output loop waits on no global load
    for (int k = tid; k < pl.P * 32; k += 256) {
        const int q = k >> 5, r = k & 31;
        const int c = r < 16 ? i0 + r : j0 + (r - 16);
        const int64_t o = (int64_t)q * KM + (c < KM ? c : 0);
        fac[k] = pl.fac_f[o];
        fac_t[k] = pl.fac_t[o];
    }
    for (int q = tid; q < pl.P; q += 256) ntr_s[q] = ll_to_float(pl.N - (pl.offs[q + 1] - pl.offs[q]));
    const int64_t seg_stride = (int64_t)pl.ntiles * TILE_ELEMS;
    const int64_t e = (int64_t)tile * TILE_ELEMS + (lj0 + ty) * TILE + (li0 + tx);
    const int32_t *hp = part_hi(pl) + e;
    const float *lp = part_lo(pl) + e;
    const int nseg = pl.nsegs;
    long long th = 0, ah = 0;
    float tl = 0.0f, al = 0.0f;
    int p = 0, p_end = pl.fold_seg[1];
    constexpr int U = 16;
    for (int g0 = 0; g0 < nseg; g0 += U) {
        int32_t h[U];
        float l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (g0 + u < nseg) {
                h[u] = __ldcs(hp + (int64_t)(g0 + u) * seg_stride);
                l[u] = __ldcs(lp + (int64_t)(g0 + u) * seg_stride);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = g0 + u;
            if (g < nseg) {
                while (g >= p_end) {   // leaving fold p (every fold holds at least one segment)
                    gh[p * 256 + tid] = ah;
                    gl[p * 256 + tid] = al;
                    th += ah;
                    tl += al;
                    ah = 0;
                    al = 0.0f;
                    ++p;
                    p_end = pl.fold_seg[p + 1];
                }
                ah += h[u];
                al += l[u];
            }
        }
    }
    gh[p * 256 + tid] = ah;
    gl[p * 256 + tid] = al;
    th += ah;
    tl += al;
    const bool cx = flags & CV_CENTER_X, cy = flags & CV_CENTER_Y;
    const bool centered = j < K ? cx : (cx || cy);
    __syncthreads();   // the staged factors
    const bool packed = pl.packed != 0;
    for (int q = 0; q < pl.P; ++q) {
        const int buf = q & 1;
        TOut *xtx = XTX ? XTX + (int64_t)q * xtx_fold_elems(pl) : nullptr;
        TOut *xty = XTY ? XTY + (int64_t)q * K * M : nullptr;
        double v = 0.0;
        if (ok) {
            const float g = ll_to_float(th - gh[q * 256 + tid]) + (tl - gl[q * 256 + tid]);
            v = entry_split_f(centered, fac[q * 32 + tx], fac[q * 32 + 16 + ty],
                              fac_t[q * 32 + tx] + fac_t[q * 32 + 16 + ty], ntr_s[q], g);
            if (j < K) {
                if (xtx && !packed) xtx[(int64_t)j * K + i] = (TOut)v;
            } else if (xty) {
                xty[(int64_t)i * M + (j - K)] = (TOut)v;
            }
        }
        vals[buf][ty][tx] = v;
        __syncthreads();
        if (xtx) {
            const int ii = i0 + ty, jj = j0 + tx;   // transposed roles: consecutive threads on consecutive jj
            if (ii < K && jj < K && (ii < jj || (packed && ii == jj)))
                xtx[packed ? packed_upper(K, ii, jj) : (int64_t)ii * K + jj] = (TOut)vals[buf][tx][ty];
        }
    }
}

template <typename TOut>
__global__ void __launch_bounds__(256, 4) k_fold_epilogue_split(const __grid_constant__ PlanView pl, int flags,
                                                             TOut *__restrict__ XTX, TOut *__restrict__ XTY) {
    grid_dep_wait();
    grid_dep_launch();
    fold_epilogue_body<TOut>(pl, flags, XTX, XTY, blockIdx.y, blockIdx.x);
}

// Batched: block per unit (problem, tile, 16 x 16 sub-tile) of the batch.
template <typename TOut>
__global__ void __launch_bounds__(256, 4) k_fold_epilogue_split_batched(const __grid_constant__ BatchTables bt,
                                                                      const __grid_constant__ BatchArgs ba) {
    grid_dep_wait();
    grid_dep_launch();
    const int4 u = bt.epi_units[blockIdx.x];
    const ProblemArgs &a = batch_arg(bt, ba, u.x);
    fold_epilogue_body<TOut>(bt.views[u.x], a.flags, (TOut *)a.XTX, (TOut *)a.XTY, u.y, u.z);
}

}  // namespace

cudaError_t shift_estimate(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y,
                           int64_t ldy, bool split, cudaStream_t st) {
    const PlanView &v = pl->v;
    ShiftArgs a;
    a.N = v.N;
    a.K = v.K;
    a.M = v.M;
    a.S = v.nsample;
    a.groups = (v.D + 31) / 32;
    a.split = split ? 1 : 0;
    a.int_bits = v.int_bits;
    a.sp = v.sp;
    a.ypack = pl->in_dtype == CV_F32 ? pl->ypack : nullptr;
    a.mp = pl->ypack_width;
    int64_t blocks = (int64_t)a.groups * SHIFT_CHUNKS;
    if (a.ypack) {   // whole clusters of packing blocks
        const int64_t pack = std::min<int64_t>((v.N + 127) / 128, (int64_t)8 * pl->num_sms);
        blocks += (pack + SHIFT_CHUNKS - 1) / SHIFT_CHUNKS * SHIFT_CHUNKS;
    }
    cudaError_t e;
    if (pl->in_dtype == CV_F32)
        e = launch_pdl(k_shift<float>, dim3((unsigned)blocks), dim3(128), 0, st, (const float *)X, ldx,
                       (const float *)Y, ldy, a);
    else
        e = launch_pdl(k_shift<double>, dim3((unsigned)blocks), dim3(128), 0, st, (const double *)X, ldx,
                       (const double *)Y, ldy, a);
    ++pl->launches;
    return e;
}

cudaError_t fold_sums(const cv_plan_s *pl, cudaStream_t st) {
    const PlanView &v = pl->v;
    const int64_t nt = (int64_t)v.ntiles * TILE_ELEMS;
    if (v.split) {
        // the total only: the statistics and the epilogue form each fold's
        // sums from its own segments' partials (fold_sum_split), so no
        // P-fold copy of H goes through memory.  The small-fold strategy
        // passes one pseudo-fold holding every segment.
        long long *th = reinterpret_cast<long long *>(v.gtot);
        ++pl->launches;
        return launch_pdl(k_fold_total_split, dim3(TILE_ELEMS / 512, v.ntiles), dim3(256), 0, st, v,
                          v.small ? 0 : v.P, th, reinterpret_cast<float *>(th + nt));
    }
    if (v.small) {
        ++pl->launches;
        return launch_pdl(k_fold_sum, dim3(TILE_ELEMS / 256, v.ntiles, 1), dim3(256), 0, st, v, 0,
                          reinterpret_cast<double *>(v.gtot));
    }
    cudaError_t e = cudaSuccess;
    for (int p0 = 0; p0 < pl->v.P && e == cudaSuccess; p0 += MAX_GRID_FOLDS) {
        const int np = std::min(MAX_GRID_FOLDS, pl->v.P - p0);
        e = launch_pdl(k_fold_sum, dim3(TILE_ELEMS / 256, pl->v.ntiles, np), dim3(256), 0, st, pl->v, p0,
                       reinterpret_cast<double *>(v.gfold));
        ++pl->launches;
    }
    if (e == cudaSuccess) e = launch_pdl(k_total_sum, dim3(TILE_ELEMS / 256, pl->v.ntiles), dim3(256), 0, st, pl->v);
    ++pl->launches;
    return e;
}

cudaError_t fold_stats(const cv_plan_s *pl, int flags, int ddof, double *mean_out, double *std_out,
                       cudaStream_t st) {
    const int KM = pl->v.K + pl->v.M;
    cudaError_t e = cudaSuccess;
    for (int p0 = pl->v.p_lo; p0 < pl->v.p_hi && e == cudaSuccess; p0 += MAX_GRID_FOLDS) {
        const int np = std::min(MAX_GRID_FOLDS, pl->v.p_hi - p0);
        e = launch_pdl(k_fold_stats, dim3((KM + 31) / 32, np), dim3(32), 0, st, pl->v, flags, ddof, mean_out,
                       std_out, p0);
        ++pl->launches;
    }
    return e;
}

bool fused_tail(const cv_plan_s *pl) {
    return pl->v.split && !pl->v.small && !pl->sharded && pl->v.P <= FOLD_SMEM_MAX;
}

cudaError_t split_stats(const cv_plan_s *pl, int flags, int ddof, double *mean_out, double *std_out, cudaStream_t st) {
    const int KM = pl->v.K + pl->v.M;
    ++pl->launches;
    return launch_pdl(k_split_stats, dim3((KM + 31) / 32, pl->v.P), dim3(32), 0, st, pl->v, flags, ddof, mean_out,
                      std_out);
}

// Dynamic shared memory of the fused fold-sum epilogue: every fold's sums of
// the block's 256 elements, its factors of the block's 16 rows and 16
// columns, their exponents, and N_T.
static size_t fold_epilogue_smem(int P) {
    return (size_t)P * (256 * (sizeof(long long) + sizeof(float)) + 32 * (sizeof(float4) + sizeof(int)) + sizeof(float));
}

cudaError_t fold_epilogue_split(const cv_plan_s *pl, int flags, void *XTX, void *XTY, cudaStream_t st) {
    const size_t smem = fold_epilogue_smem(pl->v.P);
    dim3 grid(64, pl->v.ntiles), block(16, 16);
    cudaError_t e;
    ++pl->launches;
    if (pl->out_dtype == CV_F64) {
        if ((e = cudaFuncSetAttribute(k_fold_epilogue_split<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        return launch_pdl(k_fold_epilogue_split<double>, grid, block, smem, st, pl->v, flags, (double *)XTX,
                          (double *)XTY);
    }
    if ((e = cudaFuncSetAttribute(k_fold_epilogue_split<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    return launch_pdl(k_fold_epilogue_split<float>, grid, block, smem, st, pl->v, flags, (float *)XTX, (float *)XTY);
}

cudaError_t shift_estimate_batched(const BatchTables &bt, const BatchArgs &ba, cudaStream_t st) {
    return launch_pdl(k_shift_batched, dim3((unsigned)bt.n_shift * SHIFT_CHUNKS), dim3(128), 0, st, bt, ba);
}

cudaError_t split_stats_batched(const BatchTables &bt, const BatchArgs &ba, cudaStream_t st) {
    return launch_pdl(k_split_stats_batched, dim3((unsigned)bt.n_stats), dim3(32), 0, st, bt, ba);
}

cudaError_t fold_epilogue_split_batched(const BatchTables &bt, const BatchArgs &ba, cudaStream_t st) {
    const size_t smem = fold_epilogue_smem(bt.max_P);
    cudaError_t e;
    if (bt.out_f64) {
        if ((e = cudaFuncSetAttribute(k_fold_epilogue_split_batched<double>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        return launch_pdl(k_fold_epilogue_split_batched<double>, dim3((unsigned)bt.n_epi), dim3(16, 16), smem, st, bt,
                          ba);
    }
    if ((e = cudaFuncSetAttribute(k_fold_epilogue_split_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    return launch_pdl(k_fold_epilogue_split_batched<float>, dim3((unsigned)bt.n_epi), dim3(16, 16), smem, st, bt, ba);
}

cudaError_t epilogue(const cv_plan_s *pl, int flags, void *XTX, void *XTY, cudaStream_t st) {
    dim3 block(32, 8);
    cudaError_t e = cudaSuccess;
    for (int p0 = pl->v.p_lo; p0 < pl->v.p_hi && e == cudaSuccess; p0 += MAX_GRID_FOLDS) {
        const int np = std::min(MAX_GRID_FOLDS, pl->v.p_hi - p0);
        dim3 grid((TILE / 32) * (TILE / 32), pl->v.ntiles, np);
        const bool split = pl->v.split != 0;
        if (pl->out_dtype == CV_F64)
            e = split ? launch_pdl(k_epilogue<double, true>, grid, block, 0, st, pl->v, flags, (double *)XTX,
                                   (double *)XTY, p0)
                      : launch_pdl(k_epilogue<double, false>, grid, block, 0, st, pl->v, flags, (double *)XTX,
                                   (double *)XTY, p0);
        else
            e = split ? launch_pdl(k_epilogue<float, true>, grid, block, 0, st, pl->v, flags, (float *)XTX,
                                   (float *)XTY, p0)
                      : launch_pdl(k_epilogue<float, false>, grid, block, 0, st, pl->v, flags, (float *)XTX,
                                   (float *)XTY, p0);
        ++pl->launches;
    }
    return e;
}

}  // namespace cvx
