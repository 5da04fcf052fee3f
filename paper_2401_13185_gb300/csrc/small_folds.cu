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

// Block (32 x 8 threads) per (32 x 32 sub-tile of one H tile, chunk of
// folds).  Thread (x, y) owns entries (i0 + x, j0 + y + 8 r), r < 4, keeps
// their H_R values in registers, and accumulates each fold's H_p from the
// rows staged in shared memory (up to RMAX rows of the sub-tile's 64 columns
// at a time, several small folds per stage, a large fold over several).
// When a fold's rows are done the block writes its entries: X^T X (j, i) and
// X^T Y (i, j) directly (consecutive threads on consecutive i), X^T X (i, j)
// from a shared-memory transpose, so both triangles are written coalesced and
// bitwise symmetric.
template <typename T, bool SPLIT, typename TOut>
__global__ void __launch_bounds__(256) k_epilogue_small(PlanView pl, int flags, const T *__restrict__ X, int64_t ldx,
                                                        const T *__restrict__ Y, int64_t ldy, TOut *__restrict__ XTX,
                                                        TOut *__restrict__ XTY, int fold_chunk) {
    grid_dep_wait();
    grid_dep_launch();
    using V = typename SfVal<SPLIT>::type;
    constexpr int RMAX = SPLIT ? 64 : 32;
    constexpr int FST = SPLIT ? 16 : 1;   // split path: folds whose factors a stage holds
    __shared__ V vi[RMAX][32];
    __shared__ V vj[RMAX][32];
    __shared__ double vals[2][32][33];
    __shared__ float4 fac[FST][64];
    __shared__ int fac_t[FST][64];
    __shared__ float ntr[FST];
    const int tile = blockIdx.y;
    const TileCoord tc = pl.tiles[tile];
    const int si = blockIdx.x / 4, sj = blockIdx.x % 4;
    const int li0 = si * 32, lj0 = sj * 32;
    const int i0 = tc.bi * TILE + li0, j0 = tc.bj * TILE + lj0;
    const int K = pl.K, M = pl.M, KM = K + M;
    if (i0 >= K || j0 >= KM || j0 + 31 < i0) return;
    const int p_begin = (int)blockIdx.z * fold_chunk;
    const int p_end = min(pl.P, p_begin + fold_chunk);
    if (p_begin >= p_end) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const bool cx = flags & CV_CENTER_X, cy = flags & CV_CENTER_Y;

    // H_R of my four entries
    V gr[4];
    bool ok[4];
    const int64_t nt = (int64_t)pl.ntiles * TILE_ELEMS;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int li = tx, lj = ty + 8 * r;
        const int i = i0 + li, j = j0 + lj;
        ok[r] = i < K && j < KM && i <= j;
        const int64_t it = (int64_t)tile * TILE_ELEMS + (int64_t)(lj0 + lj) * TILE + (li0 + li);
        if constexpr (SPLIT) {
            const long long *tot_hi = reinterpret_cast<const long long *>(pl.gtot);
            const float *tot_lo = reinterpret_cast<const float *>(tot_hi + nt);
            gr[r] = ll_to_float(tot_hi[it]) + tot_lo[it];
        } else {
            gr[r] = reinterpret_cast<const double *>(pl.gtot)[it];
        }
    }

    V gp[4] = {V(0), V(0), V(0), V(0)};
    int buf = 0;
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
            for (int idx = tid; idx < (pl_end - pf) * 64; idx += 256) {
                const int f = idx >> 6, q = idx & 63;
                const int c = q < 32 ? i0 + q : j0 + (q - 32);
                const int64_t o = (int64_t)(pf + f) * KM + (c < KM ? c : 0);
                fac[f][q] = pl.fac_f[o];
                fac_t[f][q] = pl.fac_t[o];
            }
            if (tid < pl_end - pf) ntr[tid] = ll_to_float(pl.N - (pl.offs[pf + tid + 1] - pl.offs[pf + tid]));
        }
        for (int idx = tid; idx < rows * 64; idx += 256) {
            const int k = idx >> 6, q = idx & 63;
            const int c = q < 32 ? i0 + q : j0 + (q - 32);
            const int64_t n = pl.perm[s0 + k];
            const V v = c < KM ? sf_value<T, SPLIT>(pl, X, ldx, Y, ldy, n, c) : V(0);
            if (q < 32)
                vi[k][q] = v;
            else
                vj[k][q - 32] = v;
        }
        __syncthreads();
        while (p < p_end && p_lo < s1) {
            const int a = (int)(max(p_lo, s0) - s0), b = (int)(min(p_hi, s1) - s0);
            for (int k = a; k < b; ++k) {
                const V x = vi[k][tx];
#pragma unroll
                for (int r = 0; r < 4; ++r) gp[r] = fma(x, vj[k][ty + 8 * r], gp[r]);
            }
            if (p_hi > s1) break;   // the fold continues in the next stage
            // fold p complete: write its entries
            TOut *xtx = XTX ? XTX + (int64_t)p * xtx_fold_elems(pl) : nullptr;
            TOut *xty = XTY ? XTY + (int64_t)p * K * M : nullptr;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int li = tx, lj = ty + 8 * r;
                const int i = i0 + li, j = j0 + lj;
                double v = 0.0;
                if (ok[r]) {
                    const bool centered = j < K ? cx : (cx || cy);
                    if constexpr (SPLIT) {
                        const int f = p - pf;
                        v = entry_split_f(centered, fac[f][li], fac[f][32 + lj], fac_t[f][li] + fac_t[f][32 + lj],
                                          ntr[f], gr[r] - gp[r]);
                    } else {
                        v = entry_f64(pl, centered, p, i, j, gr[r] - gp[r]);
                    }
                    if (j < K) {
                        if (xtx && !pl.packed) xtx[(int64_t)j * K + i] = (TOut)v;
                    } else if (xty) {
                        xty[(int64_t)i * M + (j - K)] = (TOut)v;
                    }
                }
                vals[buf][lj][li] = v;
                gp[r] = V(0);
            }
            __syncthreads();
            if (xtx) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int lj = tx, li = ty + 8 * r;
                    const int i = i0 + li, j = j0 + lj;
                    if (i < K && j < K && (i < j || (pl.packed && i == j)))
                        xtx[pl.packed ? packed_upper(K, i, j) : (int64_t)i * K + j] = (TOut)vals[buf][lj][li];
                }
            }
            buf ^= 1;
            ++p;
            if (p < p_end) {
                p_lo = p_hi;
                p_hi = pl.offs[p + 1];
            }
        }
        __syncthreads();   // the next stage overwrites vi / vj
        s0 = s1;
    }
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
    const int P = pl->v.P;
    // enough blocks to fill the GPU several times over; each block keeps its
    // 32 x 32 entries of H_R in registers across its chunk of folds
    const int64_t subtiles = (int64_t)pl->v.ntiles * 16;
    const int64_t want = (int64_t)16 * pl->num_sms;
    int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(P, (want + subtiles - 1) / subtiles));
    int fold_chunk = (int)((P + chunks - 1) / chunks);
    chunks = (P + fold_chunk - 1) / fold_chunk;
    if (chunks > MAX_GRID_FOLDS) {
        fold_chunk = (P + MAX_GRID_FOLDS - 1) / MAX_GRID_FOLDS;
        chunks = (P + fold_chunk - 1) / fold_chunk;
    }
    dim3 grid(16, pl->v.ntiles, (unsigned)chunks), block(32, 8);
    ++pl->launches;
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
