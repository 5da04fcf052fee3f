// small_folds.cu -- the small-fold strategy, for partitions whose folds hold
// only a few rows each (many folds, up to leave-one-out).
//
// The fold-grouped strategy keeps one partial tile of H = W^T W per (segment,
// tile), and a segment never straddles a fold, so with folds of ten rows it
// would pad every fold to a full k-block and move P x ntiles partial and fold
// tiles through memory.  Here instead:
//   * the contraction runs over segments that ignore fold boundaries, and only
//     H_R, H over all rows, is reduced (Algorithm 7 steps 3-4);
//   * k_small_colsums forms each fold's column sums and sums of squares from
//     its rows (steps 17, 19), which the fold statistics subtract from H_R's
//     (Lemma 14);
//   * k_epilogue_small recomputes each fold's part of every output entry,
//     H_p = W_V^T W_V, from the fold's few rows staged in shared memory, and
//     forms G_T = H_R - H_p (Lemmas 2, 3) and the centred / scaled entry in
//     the same pass (Algorithm 7 steps 8-9, 14-16, 25-27) -- no per-fold
//     scratch at all.
// Total work of the recomputation is N x (entries of one fold's outputs)
// multiply-adds, the same as a single pass of X^T [X | Y] on the CUDA cores,
// while the output writes (P x K x (K + M) values) set the pace.
//
// Values are the contraction's own: on the split path
// v = fma(x, 2^e, -s 2^e) in FP32 (the value the FP16 hi/lo pair carries, to
// within 2^-12 absolute), on the FP64 path v = x - s in FP64.
#include <algorithm>

#include "cvx_internal.cuh"

namespace cvx {
namespace {

constexpr int MAX_GRID_FOLDS = 65535;

template <bool SPLIT>
struct SfVal {
    using type = double;
};
template <>
struct SfVal<true> {
    using type = float;
};

template <typename T, bool SPLIT>
__device__ __forceinline__ typename SfVal<SPLIT>::type sf_value(const PlanView &pl, const T *__restrict__ X,
                                                                int64_t ldx, const T *__restrict__ Y, int64_t ldy,
                                                                int64_t n, int c) {
    const T x = c < pl.K ? X[n * ldx + c] : Y[n * ldy + (c - pl.K)];
    if constexpr (SPLIT) {
        if constexpr (sizeof(T) == 4) {
            const float sc = pl.sp.scale_f[c];
            return fmaf((float)x, sc, -pl.sp.shift_f[c] * sc);
        } else {
            return (float)(((double)x - pl.sp.shift[c]) * (double)pl.sp.scale_f[c]);
        }
    } else {
        return (double)x - pl.sp.shift[c];
    }
}

// Thread per (column c < K + M, fold p): the sum and the sum of squares of
// the fold's values of column c, in fold-sorted row order.
template <typename T, bool SPLIT>
__global__ void __launch_bounds__(128) k_small_colsums(PlanView pl, const T *__restrict__ X, int64_t ldx,
                                                       const T *__restrict__ Y, int64_t ldy, int p_base) {
    grid_dep_wait();
    grid_dep_launch();
    using V = typename SfVal<SPLIT>::type;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = p_base + (int)blockIdx.y;
    const int KM = pl.K + pl.M;
    if (c >= KM) return;
    const int64_t r0 = pl.offs[p], r1 = pl.offs[p + 1];
    V s = V(0), q = V(0);
    for (int64_t r = r0; r < r1; ++r) {
        const V v = sf_value<T, SPLIT>(pl, X, ldx, Y, ldy, pl.perm[r], c);
        s += v;
        q = fma(v, v, q);
    }
    if constexpr (SPLIT)
        reinterpret_cast<float2 *>(pl.fold_sq)[(int64_t)p * KM + c] = make_float2(s, q);
    else
        reinterpret_cast<double2 *>(pl.fold_sq)[(int64_t)p * KM + c] = make_double2(s, q);
}

// Block (16 x 16 threads) per (64 x 64 output tile, chunk of folds).  X^T X
// tiles (bi, bj), bi <= bj, cover rows i0 = 64 bi and columns j0 = 64 bj of
// X^T X; X^T Y tiles cover rows i0 and 64 of Y's columns.  Thread (x, y)
// owns the 4 x 4 entries (i0 + 4 y + a, j0 + 4 x + u), keeps their H_R
// values in registers, and accumulates each fold's H_p from the rows staged
// in shared memory (up to RMAX rows of the tile's 128 columns at a time,
// several small folds per stage, a large fold over several): two 16-byte
// shared loads and 16 multiply-adds per row.  When a fold's rows are done the
// thread writes its entries as 4 runs of 4 consecutive values (one 32-byte
// sector each for FP64) and, for an off-diagonal X^T X tile, their mirror
// (j, i) the same way, so no transpose passes through shared memory.  Entry
// (i, j) and its mirror come from the same operands in the same order (the
// upper-triangle H_R entry, the fold's products over the same rows, the
// per-column factors in the order (min, max)), so the two triangles are
// bitwise symmetric.  A packed upper-triangle output takes the entries with
// i <= j only.
constexpr int SF_T = 64;     // output tile edge
constexpr int SF_FST = 8;    // split path: folds whose factors a stage holds

// Split path: a thread's 4 x 4 entries of fold p from G_T = H_R - H_p (gr -
// gp) and the fold's per-column factors of its rows (fi, ti) and columns
// (fj, tj), with the factors taken in the order (min, max) of the entry's
// indices (Propositions 7, 8, 15, 16).  Off the diagonal (DIAG false) every
// row index is below every column index.
template <typename TOut, bool DIAG>
__device__ __forceinline__ void split_entries(const float (&gr)[4][4], const float (&gp)[4][4], const float4 *fi,
                                              const int *ti, const float4 *fj, const int *tj, int ib, int jb,
                                              bool centered, float ntr, TOut (&out)[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const float4 fa = fi[a];
        const int ta = ti[a];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 fb = fj[u];
            const int tb = tj[u];
            const bool up = !DIAG || ib + a <= jb + u;
            const float g = gr[a][u] - gp[a][u];
            const float aa = fa.x * fb.x;
            const float4 &f1 = up ? fa : fb;
            const float4 &f2 = up ? fb : fa;
            const float r = centered ? fmaf(g, aa, -f1.y * f2.z)
                                     : fmaf(g, aa, fmaf(f1.w, f2.y, fmaf(f1.y, f2.w, ntr * f1.w * f2.w)));
            out[a][u] = scaled_out<TOut>(r, ta + tb);
        }
    }
}

// A thread's entries of fold p into the outputs: X^T Y rows, or X^T X rows as
// 4-value runs and, for an off-diagonal tile, their mirror (j, i) the same
// way; the packed layout takes the upper entries one by one.
template <typename TOut>
__device__ __forceinline__ void store_fold(const PlanView &pl, int p, const TOut (&out)[4][4], const bool (&ok)[4][4],
                                           int ib, int jb, bool ytile, bool diag, bool vec_row, bool vec_mir,
                                           TOut *__restrict__ XTX, TOut *__restrict__ XTY) {
    const int K = pl.K, M = pl.M;
    if (ytile) {
        if (XTY) {
            TOut *xty = XTY + (int64_t)p * K * M;
#pragma unroll
            for (int a = 0; a < 4; ++a)
                if (ib + a < K) store4(xty + (int64_t)(ib + a) * M + (jb - K), out[a], vec_row, ok[a]);
        }
    } else if (XTX) {
        TOut *xtx = XTX + (int64_t)p * xtx_fold_elems(pl);
        if (pl.packed) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (ok[a][u]) xtx[packed_upper(K, ib + a, jb + u)] = out[a][u];
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a)
                if (ib + a < K) store4(xtx + (int64_t)(ib + a) * K + jb, out[a], vec_row, ok[a]);
            if (!diag) {   // the mirror (j, i): column u of my entries is a run along row jb + u
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (jb + u < K) {
                        const TOut m4[4] = {out[0][u], out[1][u], out[2][u], out[3][u]};
                        const bool okm[4] = {ok[0][u], ok[1][u], ok[2][u], ok[3][u]};
                        store4(xtx + (int64_t)(jb + u) * K + ib, m4, vec_mir, okm);
                    }
                }
            }
        }
    }
}

template <typename T, bool SPLIT, typename TOut>
__global__ void __launch_bounds__(256, SPLIT ? 3 : 1) k_epilogue_small(PlanView pl, int flags, const T *__restrict__ X, int64_t ldx,
                                                        const T *__restrict__ Y, int64_t ldy, TOut *__restrict__ XTX,
                                                        TOut *__restrict__ XTY, int fold_chunk) {
    grid_dep_wait();
    grid_dep_launch();
    using V = typename SfVal<SPLIT>::type;
    constexpr int RMAX = SPLIT ? 64 : 32;
    constexpr int FST = SPLIT ? SF_FST : 1;
    __shared__ __align__(16) V vi[RMAX][SF_T];
    __shared__ __align__(16) V vj[RMAX][SF_T];
    __shared__ float4 fac_i[FST][SF_T], fac_j[FST][SF_T];
    __shared__ int ft_i[FST][SF_T], ft_j[FST][SF_T];
    __shared__ float ntr[FST];
    __shared__ int64_t offs_s[FST + 1];   // split path: the stage's fold boundaries
    const int K = pl.K, M = pl.M, KM = K + M;
    const int nx = (K + SF_T - 1) / SF_T;
    const int bi = (int)blockIdx.x, by = (int)blockIdx.y;
    const bool ytile = by >= nx;   // an X^T Y tile
    if (!ytile && by < bi) return;
    const int i0 = bi * SF_T;
    const int j0 = ytile ? K + (by - nx) * SF_T : by * SF_T;   // first column of W
    const int jlim = ytile ? KM : K;
    const bool diag = !ytile && by == bi;
    const bool packed = pl.packed != 0;
    const int p_begin = (int)blockIdx.z * fold_chunk;
    const int p_end = min(pl.P, p_begin + fold_chunk);
    if (p_begin >= p_end) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
    const bool cx = flags & CV_CENTER_X, cy = flags & CV_CENTER_Y;
    const bool centered = ytile ? (cx || cy) : cx;
    const int ib = i0 + 4 * ty, jb = j0 + 4 * tx;   // my first row and column

    // H_R of my entries, from the upper block triangle of tiles: entry (a, b),
    // a <= b, at element (b % TILE) * TILE + a % TILE of tile (a / TILE, b / TILE)
    V gr[4][4];
    bool ok[4][4];
    const int64_t nt = (int64_t)pl.ntiles * TILE_ELEMS;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = ib + a, j = jb + u;
            ok[a][u] = i < K && j < jlim && (!packed || i <= j);
            gr[a][u] = V(0);
            if (i < K && j < jlim) {
                const int lo = min(i, j), hi = max(i, j);
                const int64_t it = (int64_t)tile_index(pl.nb, lo / TILE, hi / TILE) * TILE_ELEMS +
                                   (int64_t)(hi % TILE) * TILE + (lo % TILE);
                if constexpr (SPLIT) {
                    const long long *tot_hi = reinterpret_cast<const long long *>(pl.gtot);
                    const float *tot_lo = reinterpret_cast<const float *>(tot_hi + nt);
                    gr[a][u] = ll_to_float(tot_hi[it]) + tot_lo[it];
                } else {
                    gr[a][u] = reinterpret_cast<const double *>(pl.gtot)[it];
                }
            }
        }
    }
    // whole 4-value runs go out as one vector store when they are aligned
    const uintptr_t vbytes = 4 * sizeof(TOut);
    const bool aligned = ytile ? (uintptr_t)XTY % vbytes == 0 : (uintptr_t)XTX % vbytes == 0;
    const bool vec_row = aligned && !packed && (ytile ? (M % 4 == 0) : (K % 4 == 0)) && jb + 3 < jlim;
    const bool vec_mir = aligned && !packed && K % 4 == 0 && ib + 3 < K;

    V gp[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int u = 0; u < 4; ++u) gp[a][u] = V(0);
    int p = p_begin;
    int64_t p_lo = pl.offs[p], p_hi = pl.offs[p + 1];   // rows of fold p
    const int64_t r_all = pl.offs[p_end];
    for (int64_t s0 = p_lo; s0 < r_all;) {
        // split path: a stage also ends before the fold FST after the one
        // holding row s0, so its factors fit the staged table
        const int pf = p;
        const int pl_end = SPLIT ? min(p_end, pf + FST) : p_end;
        const int64_t s1 = min(min(s0 + (int64_t)RMAX, r_all), (int64_t)pl.offs[pl_end]);
        const int rows = (int)(s1 - s0);
        if constexpr (SPLIT) {
            for (int idx = tid; idx < (pl_end - pf) * 2 * SF_T; idx += 256) {
                const int f = idx / (2 * SF_T), q = idx % (2 * SF_T);
                const int c = q < SF_T ? i0 + q : j0 + (q - SF_T);
                const int64_t o = (int64_t)(pf + f) * KM + (c < KM ? c : 0);
                if (q < SF_T) {
                    fac_i[f][q] = pl.fac_f[o];
                    ft_i[f][q] = pl.fac_t[o];
                } else {
                    fac_j[f][q - SF_T] = pl.fac_f[o];
                    ft_j[f][q - SF_T] = pl.fac_t[o];
                }
            }
            if (tid < pl_end - pf) ntr[tid] = ll_to_float(pl.N - (pl.offs[pf + tid + 1] - pl.offs[pf + tid]));
            if (tid <= pl_end - pf) offs_s[tid] = pl.offs[pf + tid];
        }
        for (int idx = tid; idx < rows * 2 * SF_T; idx += 256) {
            const int k = idx / (2 * SF_T), q = idx % (2 * SF_T);
            const int c = q < SF_T ? i0 + q : j0 + (q - SF_T);
            const int64_t n = pl.perm[s0 + k];
            const V v = c < (q < SF_T ? K : jlim) ? sf_value<T, SPLIT>(pl, X, ldx, Y, ldy, n, c) : V(0);
            if (q < SF_T)
                vi[k][q] = v;
            else
                vj[k][q - SF_T] = v;
        }
        __syncthreads();
        while (p < p_end && p_lo < s1) {
            const int ka = (int)(max(p_lo, s0) - s0), kb = (int)(min(p_hi, s1) - s0);
            for (int k = ka; k < kb; ++k) {
                V xi[4], xj[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) xi[a] = vi[k][4 * ty + a];
#pragma unroll
                for (int u = 0; u < 4; ++u) xj[u] = vj[k][4 * tx + u];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int u = 0; u < 4; ++u) gp[a][u] = fma(xi[a], xj[u], gp[a][u]);
            }
            if (p_hi > s1) break;   // the fold continues in the next stage
            // fold p complete: its entries
            TOut out[4][4];
            if constexpr (SPLIT) {
                const int f = p - pf;
                float4 fi[4], fj[4];
                int ti[4], tj[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    fi[a] = fac_i[f][4 * ty + a];
                    ti[a] = ft_i[f][4 * ty + a];
                    fj[a] = fac_j[f][4 * tx + a];
                    tj[a] = ft_j[f][4 * tx + a];
                }
                if (diag)
                split_entries<TOut, true>(gr, gp, fi, ti, fj, tj, ib, jb, centered, ntr[f], out);
            else
                split_entries<TOut, false>(gr, gp, fi, ti, fj, tj, ib, jb, centered, ntr[f], out);
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = ib + a, j = jb + u;
                        out[a][u] = ok[a][u] ? (TOut)entry_f64(pl, centered, p, min(i, j), max(i, j),
                                                               gr[a][u] - gp[a][u])
                                             : TOut(0);
                    }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int u = 0; u < 4; ++u) gp[a][u] = V(0);
            store_fold<TOut>(pl, p, out, ok, ib, jb, ytile, diag, vec_row, vec_mir, XTX, XTY);
            ++p;
            if (p < p_end) {
                p_lo = p_hi;
                // split path: the stage holds the boundaries of its folds (p < pl_end here, or the loop ends)
                p_hi = SPLIT && p < pl_end ? offs_s[p + 1 - pf] : pl.offs[p + 1];
            }
        }
        __syncthreads();   // the next stage overwrites the staged rows and factors
        s0 = s1;
    }
}

// Split path with FP32 inputs: the same epilogue with its staging double
// buffered, so that the copies of a stage's rows and factors are in flight
// while the block computes the previous stage.  Each buffer holds SP_RMAX
// rows of the tile's 128 columns, the factors of up to SP_FST folds and their
// boundaries; the copies are asynchronous (cp.async), and each thread
// converts the row values it copied itself (its column is fixed: tid % 128)
// once they have landed, before the block barrier.  Columns past the
// problem's are never copied and stay zero.  The arithmetic is that of
// k_epilogue_small.
constexpr int SP_RMAX = 64;
constexpr int SP_FST = 8;

struct __align__(16) SfStage {
    float v[SP_RMAX][2 * SF_T];   // row values: columns i0 .. i0 + 63, then j0 .. j0 + 63
    float4 fac[SP_FST][2 * SF_T];
    int ft[SP_FST][2 * SF_T];
    long long offs[SP_FST + 1];
};
constexpr size_t SP_SMEM = 2 * sizeof(SfStage);

__device__ __forceinline__ void cpa4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Rows [s0, s1) and folds [pf, pe) of one stage: pf holds row s0, pe is at
// most SP_FST folds further, and the stage ends at the first of RMAX rows,
// the block's last row and the first row of fold pe.
struct SpStage {
    int64_t s0, s1;
    int pf, pe;
};

__device__ __forceinline__ SpStage sp_stage(const PlanView &pl, int64_t s0, int pf, int p_end, int64_t r_all) {
    while (pl.offs[pf + 1] <= s0) ++pf;
    SpStage g;
    g.s0 = s0;
    g.pf = pf;
    g.pe = min(p_end, pf + SP_FST);
    g.s1 = min(min(s0 + (int64_t)SP_RMAX, r_all), (int64_t)pl.offs[g.pe]);
    return g;
}

template <typename TOut>
__global__ void __launch_bounds__(256, 2) k_epilogue_small_pipe(PlanView pl, int flags, const float *__restrict__ X,
                                                                int64_t ldx, const float *__restrict__ Y, int64_t ldy,
                                                                TOut *__restrict__ XTX, TOut *__restrict__ XTY,
                                                                int fold_chunk) {
    grid_dep_wait();
    grid_dep_launch();
    extern __shared__ __align__(16) uint8_t sp_raw[];
    SfStage *buf = reinterpret_cast<SfStage *>(sp_raw);
    const int K = pl.K, M = pl.M, KM = K + M;
    const int nx = (K + SF_T - 1) / SF_T;
    const int bi = (int)blockIdx.x, by = (int)blockIdx.y;
    const bool ytile = by >= nx;
    if (!ytile && by < bi) return;
    const int i0 = bi * SF_T;
    const int j0 = ytile ? K + (by - nx) * SF_T : by * SF_T;
    const int jlim = ytile ? KM : K;
    const bool diag = !ytile && by == bi;
    const bool packed = pl.packed != 0;
    const int p_begin = (int)blockIdx.z * fold_chunk;
    const int p_end = min(pl.P, p_begin + fold_chunk);
    if (p_begin >= p_end) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
    const bool cx = flags & CV_CENTER_X, cy = flags & CV_CENTER_Y;
    const bool centered = ytile ? (cx || cy) : cx;
    const int ib = i0 + 4 * ty, jb = j0 + 4 * tx;

    float gr[4][4];
    bool ok[4][4];
    const int64_t nt = (int64_t)pl.ntiles * TILE_ELEMS;
    const long long *tot_hi = reinterpret_cast<const long long *>(pl.gtot);
    const float *tot_lo = reinterpret_cast<const float *>(tot_hi + nt);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = ib + a, j = jb + u;
            ok[a][u] = i < K && j < jlim && (!packed || i <= j);
            gr[a][u] = 0.0f;
            if (i < K && j < jlim) {
                const int lo = min(i, j), hi = max(i, j);
                const int64_t it = (int64_t)tile_index(pl.nb, lo / TILE, hi / TILE) * TILE_ELEMS +
                                   (int64_t)(hi % TILE) * TILE + (lo % TILE);
                gr[a][u] = ll_to_float(tot_hi[it]) + tot_lo[it];
            }
        }
    }
    const uintptr_t vbytes = 4 * sizeof(TOut);
    const bool aligned = ytile ? (uintptr_t)XTY % vbytes == 0 : (uintptr_t)XTX % vbytes == 0;
    const bool vec_row = aligned && !packed && (ytile ? (M % 4 == 0) : (K % 4 == 0)) && jb + 3 < jlim;
    const bool vec_mir = aligned && !packed && K % 4 == 0 && ib + 3 < K;

    // this thread's staged column (the same in every stage) and its conversion
    const int q = tid % (2 * SF_T), k_first = tid / (2 * SF_T);
    const int col = q < SF_T ? i0 + q : j0 + (q - SF_T);
    const bool live = col < (q < SF_T ? K : jlim);
    const float sc = live ? pl.sp.scale_f[col] : 0.0f;
    const float ns = live ? -pl.sp.shift_f[col] * sc : 0.0f;
    const float *src = col < K ? X + col : Y + (col - K);
    const int64_t ld = col < K ? ldx : ldy;
    if (!live)
        for (int k = k_first; k < SP_RMAX; k += 256 / (2 * SF_T)) buf[0].v[k][q] = buf[1].v[k][q] = 0.0f;

    auto issue = [&](const SpStage &g, SfStage &b) {
        for (int idx = tid; idx < (g.pe - g.pf) * 2 * SF_T; idx += 256) {
            const int f = idx / (2 * SF_T), qq = idx % (2 * SF_T);
            const int c = qq < SF_T ? i0 + qq : j0 + (qq - SF_T);
            const int64_t o = (int64_t)(g.pf + f) * KM + (c < KM ? c : 0);
            cpa16(&b.fac[f][qq], &pl.fac_f[o]);
            cpa4(&b.ft[f][qq], &pl.fac_t[o]);
        }
        if (tid <= g.pe - g.pf) cpa8(&b.offs[tid], &pl.offs[g.pf + tid]);
        if (live)
            for (int k = k_first; k < (int)(g.s1 - g.s0); k += 256 / (2 * SF_T))
                cpa4(&b.v[k][q], src + (int64_t)pl.perm[g.s0 + k] * ld);
    };

    float gp[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int u = 0; u < 4; ++u) gp[a][u] = 0.0f;
    const int64_t r_all = pl.offs[p_end];
    int p = p_begin;
    int64_t p_lo = pl.offs[p], p_hi = pl.offs[p + 1];
    SpStage cur = sp_stage(pl, p_lo, p_begin, p_end, r_all);
    issue(cur, buf[0]);
    cpa_commit();
    for (int t = 0; cur.s0 < r_all; ++t) {
        SfStage &b = buf[t & 1];
        const bool more = cur.s1 < r_all;
        SpStage nxt = cur;
        if (more) {
            nxt = sp_stage(pl, cur.s1, cur.pf, p_end, r_all);
            issue(nxt, buf[(t + 1) & 1]);
        }
        cpa_commit();
        cpa_wait<1>();   // this thread's copies of the current stage have landed
        if (live)
            for (int k = k_first; k < (int)(cur.s1 - cur.s0); k += 256 / (2 * SF_T)) b.v[k][q] = fmaf(b.v[k][q], sc, ns);
        __syncthreads();
        while (p < p_end && p_lo < cur.s1) {
            const int ka = (int)(max(p_lo, cur.s0) - cur.s0), kb = (int)(min(p_hi, cur.s1) - cur.s0);
            for (int k = ka; k < kb; ++k) {
                const float4 xi = *reinterpret_cast<const float4 *>(&b.v[k][4 * ty]);
                const float4 xj = *reinterpret_cast<const float4 *>(&b.v[k][SF_T + 4 * tx]);
                const float xa[4] = {xi.x, xi.y, xi.z, xi.w}, xu[4] = {xj.x, xj.y, xj.z, xj.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int u = 0; u < 4; ++u) gp[a][u] = fmaf(xa[a], xu[u], gp[a][u]);
            }
            if (p_hi > cur.s1) break;   // the fold continues in the next stage
            const int f = p - cur.pf;
            float4 fi[4], fj[4];
            int ti[4], tj[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                fi[a] = b.fac[f][4 * ty + a];
                ti[a] = b.ft[f][4 * ty + a];
                fj[a] = b.fac[f][SF_T + 4 * tx + a];
                tj[a] = b.ft[f][SF_T + 4 * tx + a];
            }
            const float ntr = ll_to_float(pl.N - (b.offs[f + 1] - b.offs[f]));
            TOut out[4][4];
            if (diag)
                split_entries<TOut, true>(gr, gp, fi, ti, fj, tj, ib, jb, centered, ntr, out);
            else
                split_entries<TOut, false>(gr, gp, fi, ti, fj, tj, ib, jb, centered, ntr, out);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int u = 0; u < 4; ++u) gp[a][u] = 0.0f;
            store_fold<TOut>(pl, p, out, ok, ib, jb, ytile, diag, vec_row, vec_mir, XTX, XTY);
            ++p;
            if (p < p_end) {
                p_lo = p_hi;
                p_hi = p < cur.pe ? b.offs[p + 1 - cur.pf] : pl.offs[p + 1];
            }
        }
        __syncthreads();   // the next issue overwrites this buffer
        cur = nxt;
        if (!more) break;
    }
    cpa_wait<0>();
}

template <typename T, bool SPLIT>
cudaError_t launch_colsums(const cv_plan_s *pl, const T *X, int64_t ldx, const T *Y, int64_t ldy, cudaStream_t st) {
    const int KM = pl->v.K + pl->v.M;
    cudaError_t e = cudaSuccess;
    for (int p0 = 0; p0 < pl->v.P && e == cudaSuccess; p0 += MAX_GRID_FOLDS) {
        const int np = std::min(MAX_GRID_FOLDS, pl->v.P - p0);
        e = launch_pdl(k_small_colsums<T, SPLIT>, dim3((KM + 127) / 128, np), dim3(128), 0, st, pl->v, X, ldx, Y,
                       ldy, p0);
        ++pl->launches;
    }
    return e;
}

template <typename T, bool SPLIT>
cudaError_t launch_epilogue(const cv_plan_s *pl, int flags, const T *X, int64_t ldx, const T *Y, int64_t ldy,
                            void *XTX, void *XTY, cudaStream_t st) {
    const int P = pl->v.P, nx = (pl->v.K + SF_T - 1) / SF_T, ny = (pl->v.M + SF_T - 1) / SF_T;
    // enough blocks to fill the GPU several times over; each block keeps its
    // 64 x 64 entries of H_R in registers across its chunk of folds
    const int64_t subtiles = (int64_t)nx * (nx + 1) / 2 + (int64_t)nx * ny;
    const int64_t want = (int64_t)16 * pl->num_sms;
    int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(P, (want + subtiles - 1) / subtiles));
    int fold_chunk = (int)((P + chunks - 1) / chunks);
    chunks = (P + fold_chunk - 1) / fold_chunk;
    if (chunks > MAX_GRID_FOLDS) {
        fold_chunk = (P + MAX_GRID_FOLDS - 1) / MAX_GRID_FOLDS;
        chunks = (P + fold_chunk - 1) / fold_chunk;
    }
    dim3 grid((unsigned)nx, (unsigned)(nx + ny), (unsigned)chunks), block(16, 16);
    ++pl->launches;
    // as much of the SM's on-chip memory as shared memory as it takes, so
    // that the blocks resident per SM are not limited by it
    cudaError_t e = cudaFuncSetAttribute(k_epilogue_small<T, SPLIT, double>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_epilogue_small<T, SPLIT, float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 100);
    if (e != cudaSuccess) return e;
    if constexpr (SPLIT && sizeof(T) == sizeof(float)) {
        const float *x = (const float *)X, *y = (const float *)Y;
        if (pl->out_dtype == CV_F64) {
            e = cudaFuncSetAttribute(k_epilogue_small_pipe<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SP_SMEM);
            if (e != cudaSuccess) return e;
            return launch_pdl(k_epilogue_small_pipe<double>, grid, block, SP_SMEM, st, pl->v, flags, x, ldx, y, ldy,
                              (double *)XTX, (double *)XTY, fold_chunk);
        }
        e = cudaFuncSetAttribute(k_epilogue_small_pipe<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SP_SMEM);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_epilogue_small_pipe<float>, grid, block, SP_SMEM, st, pl->v, flags, x, ldx, y, ldy,
                          (float *)XTX, (float *)XTY, fold_chunk);
    }
    if (pl->out_dtype == CV_F64)
        return launch_pdl(k_epilogue_small<T, SPLIT, double>, grid, block, 0, st, pl->v, flags, X, ldx, Y, ldy,
                          (double *)XTX, (double *)XTY, fold_chunk);
    return launch_pdl(k_epilogue_small<T, SPLIT, float>, grid, block, 0, st, pl->v, flags, X, ldx, Y, ldy,
                      (float *)XTX, (float *)XTY, fold_chunk);
}

}  // namespace

cudaError_t small_fold_colsums(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                               cudaStream_t st) {
    const bool split = pl->v.split != 0;
    if (pl->in_dtype == CV_F32) {
        const float *x = (const float *)X, *y = (const float *)Y;
        return split ? launch_colsums<float, true>(pl, x, ldx, y, ldy, st)
                     : launch_colsums<float, false>(pl, x, ldx, y, ldy, st);
    }
    const double *x = (const double *)X, *y = (const double *)Y;
    return split ? launch_colsums<double, true>(pl, x, ldx, y, ldy, st)
                 : launch_colsums<double, false>(pl, x, ldx, y, ldy, st);
}

cudaError_t small_fold_epilogue(const cv_plan_s *pl, int flags, const void *X, int64_t ldx, const void *Y,
                                int64_t ldy, void *XTX, void *XTY, cudaStream_t st) {
    const bool split = pl->v.split != 0;
    if (pl->in_dtype == CV_F32) {
        const float *x = (const float *)X, *y = (const float *)Y;
        return split ? launch_epilogue<float, true>(pl, flags, x, ldx, y, ldy, XTX, XTY, st)
                     : launch_epilogue<float, false>(pl, flags, x, ldx, y, ldy, XTX, XTY, st);
    }
    const double *x = (const double *)X, *y = (const double *)Y;
    return split ? launch_epilogue<double, true>(pl, flags, x, ldx, y, ldy, XTX, XTY, st)
                 : launch_epilogue<double, false>(pl, flags, x, ldx, y, ldy, XTX, XTY, st);
}

}  // namespace cvx
