// ridge.cu -- per-fold ridge regression / OLS on the products, and the
// models' squared error on each validation partition.
//
// The paper names ridge regression and OLS through the normal equations as
// consumers of X^T X and X^T Y, and cross-validation as fitting on each
// training partition and evaluating on its validation partition (Section 1).
//
//   cv_ridge        For each fold p, B_p = (XTX_p + lambda I)^-1 XTY_p by the
//                   Cholesky factorisation XTX_p + lambda I = L L^T in FP64
//                   (blocked, every fold's blocks in the same launches), then
//                   forward and back substitution by a cluster of blocks per
//                   fold.
//   cv_ridge_press  press[p][m] = sum over the validation rows n of fold p of
//                   (y_nm - y^_nm)^2.  Each validation row is preprocessed
//                   with its fold's TRAINING statistics (x~ = (x - [cX] mean)
//                   / ([sX] ? std : 1)), predicted in that space (x~ B_p) and
//                   mapped back to Y's units (times [sY] std, plus [cY] mean).
//
// All arithmetic is FP64, and the FP64 pipe bounds both calls: K^3 / 6
// multiply-adds per fold for the factorisation's trailing updates, N K M for
// the predictions.
#include <math.h>

#include <cooperative_groups.h>

#include <algorithm>

#include "cvx_internal.cuh"

namespace cvx {
namespace {

namespace cg = cooperative_groups;

constexpr int PRESS_THREADS = 256;
constexpr int PRESS_WARPS = PRESS_THREADS / 32;
constexpr int PRESS_MC = 16;                      // responses per pass over a row
constexpr size_t PRESS_SMEM_TARGET = 100 * 1024;  // two blocks per SM when it fits
constexpr size_t PRESS_SMEM_MAX = 200 * 1024;

// Blocked right-looking Cholesky, all folds at once, RB x RB blocks (FP64).
// The factor is built in place in the caller's workspace L, row-major per
// fold (L[i K + j], j <= i; the strict upper triangle is zero).  Launches:
//   k_ridge_init    L = lower triangle of XTX + lambda I, info = 0;
//   k_ridge_potrf   factors the first diagonal block;
// then for each block column b with blocks below it:
//   k_ridge_trsm    each block below the diagonal: X L_bb^T = A_ib,b by
//                   forward substitution, a warp per row;
//   k_ridge_update  each trailing block (ib >= kb > b): A_ib,kb -=
//                   L_ib,b L_kb,b^T; the block that finishes diagonal block
//                   b + 1 factors it as well, so it is ready for the next
//                   column's trsm.
// A diagonal block is factored by one thread block in shared memory.  A
// pivot that is not positive records info[p] = j + 1 (the global column)
// and stops the fold.  The sums run in another order than a column-by-column
// factorisation, so results agree to rounding.
constexpr int RB = 32;
constexpr int LD_STRIDE = RB + 1;

__global__ void __launch_bounds__(256) k_ridge_init(int K, const double *__restrict__ XTX, double lambda,
                                                    double *__restrict__ L, int32_t *__restrict__ info) {
    grid_dep_wait();
    grid_dep_launch();
    const int p = blockIdx.y;
    const int64_t KK = (int64_t)K * K;
    const double *A = XTX + p * KK;
    double *Lp = L + p * KK;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < KK; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / K), j = (int)(e % K);
        Lp[e] = j <= i ? A[e] + (i == j ? lambda : 0.0) : 0.0;   // only the lower triangle is read
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) info[p] = 0;
}

// The block's threads factor the nb x nb lower triangle held in D (row
// stride LD_STRIDE) in place, right-looking: per column j, the pivot's
// reciprocal r = rsqrt(d_jj) (l_jj = d_jj r), the column below it scaled by
// r, then the trailing triangle updated.  Returns, in every thread, 0 or
// the failing local column + 1.  Uses the caller's shared scalars.
__device__ int factor_diag_block(double *D, int nb, double *r_sh, int *fail_sh) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < nb; ++j) {
        if (tid == 0) {
            const double d2 = D[j * LD_STRIDE + j];
            if (d2 > 0.0) {
                const double r = rsqrt(d2);
                D[j * LD_STRIDE + j] = d2 * r;
                *r_sh = r;
                *fail_sh = 0;
            } else {
                *fail_sh = j + 1;
            }
        }
        __syncthreads();
        if (*fail_sh) return *fail_sh;
        const double r = *r_sh;
        for (int i = j + 1 + tid; i < nb; i += nt) D[i * LD_STRIDE + j] *= r;
        __syncthreads();
        // the trailing triangle j < k <= i < nb (m = nb - 1 - j rows), its
        // m (m + 1) / 2 entries enumerated row by row: entry e is (ii, kk) with
        // ii (ii + 1) / 2 <= e < (ii + 1) (ii + 2) / 2, so that every issued
        // multiply-add is a useful one
        const int m = nb - 1 - j;
        for (int e = tid; e < m * (m + 1) / 2; e += nt) {
            int ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            if ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
            if (ii * (ii + 1) / 2 > e) --ii;
            const int i = j + 1 + ii, k = j + 1 + (e - ii * (ii + 1) / 2);
            D[i * LD_STRIDE + k] = fma(-D[i * LD_STRIDE + j], D[k * LD_STRIDE + j], D[i * LD_STRIDE + k]);
        }
        __syncthreads();
    }
    return 0;
}

__global__ void __launch_bounds__(256) k_ridge_potrf(int K, double *__restrict__ L, int32_t *__restrict__ info) {
    grid_dep_wait();
    grid_dep_launch();
    const int p = blockIdx.x, tid = threadIdx.x;
    if (info[p] != 0) return;
    __shared__ double D[RB * LD_STRIDE];
    __shared__ double r_sh;
    __shared__ int fail_sh;
    const int nb = min(RB, K);
    double *Lp = L + (int64_t)p * K * K;
    for (int e = tid; e < RB * RB; e += blockDim.x) {
        const int i = e / RB, j = e % RB;
        D[i * LD_STRIDE + j] = (i < nb && j <= i) ? Lp[(int64_t)i * K + j] : 0.0;
    }
    __syncthreads();
    const int fail = factor_diag_block(D, nb, &r_sh, &fail_sh);
    if (fail) {
        if (tid == 0) info[p] = fail;
        return;
    }
    for (int e = tid; e < RB * RB; e += blockDim.x) {
        const int i = e / RB, j = e % RB;
        if (i < nb && j <= i) Lp[(int64_t)i * K + j] = D[i * LD_STRIDE + j];
    }
}

// Block (block row ib > b, fold); a warp per TRSM_ROWS rows of the block.
// Row i: x L_bb^T = a, right-looking: once a_j is final, a_k -= a_j (l_kj /
// l_jj) for k > j (the columns of L_bb scaled once per block), and x_k =
// a_k / l_kk at the end; lane k holds a_k.  The warp's rows run
// interleaved.
constexpr int TRSM_THREADS = 256;
constexpr int TRSM_ROWS = RB / (TRSM_THREADS / 32);

__global__ void __launch_bounds__(TRSM_THREADS) k_ridge_trsm(int K, int r0, double *__restrict__ L,
                                                             const int32_t *__restrict__ info) {
    grid_dep_wait();
    grid_dep_launch();
    const int p = blockIdx.y, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (info[p] != 0) return;
    __shared__ double Lb[RB * LD_STRIDE];
    __shared__ double inv[RB];
    const int nb = min(RB, K - r0);
    const int i0 = r0 + RB * (1 + (int)blockIdx.x) + w * TRSM_ROWS;   // the warp's first row
    double *Lp = L + (int64_t)p * K * K;
    for (int e = tid; e < RB * RB; e += TRSM_THREADS) {
        const int i = e / RB, j = e % RB;
        Lb[i * LD_STRIDE + j] = (i < nb && j <= i) ? Lp[(int64_t)(r0 + i) * K + r0 + j] : 0.0;
    }
    __syncthreads();
    if (tid < nb) inv[tid] = 1.0 / Lb[tid * LD_STRIDE + tid];
    __syncthreads();
    for (int e = tid; e < RB * RB; e += TRSM_THREADS) {   // column j scaled by 1 / l_jj
        const int i = e / RB, j = e % RB;
        if (j < i) Lb[i * LD_STRIDE + j] *= inv[j];
    }
    __syncthreads();
    double a[TRSM_ROWS];
#pragma unroll
    for (int t = 0; t < TRSM_ROWS; ++t) {
        const int i = i0 + t;
        a[t] = (i < K && lane < nb) ? Lp[(int64_t)i * K + r0 + lane] : 0.0;
    }
    // a_k -= a_j l_kj / l_jj once a_j is final; x_k = a_k / l_kk at the end
    for (int j = 0; j < nb; ++j) {
        const double skj = Lb[lane * LD_STRIDE + j];
#pragma unroll
        for (int t = 0; t < TRSM_ROWS; ++t) {
            const double aj = __shfl_sync(0xffffffffu, a[t], j);
            if (lane > j) a[t] = fma(-aj, skj, a[t]);
        }
    }
    const double il = lane < nb ? inv[lane] : 0.0;
#pragma unroll
    for (int t = 0; t < TRSM_ROWS; ++t) {
        const int i = i0 + t;
        if (i < K && lane < nb) Lp[(int64_t)i * K + r0 + lane] = a[t] * il;
    }
}

// Block (trailing block (ib, kb), b < kb <= ib, fold): L_ib,kb -= L_ib,b
// L_kb,b^T (lower entries only on the diagonal blocks).  The block of
// diagonal block b + 1 then factors it.
__global__ void __launch_bounds__(256) k_ridge_update(int K, int r0, double *__restrict__ L,
                                                      int32_t *__restrict__ info) {
    grid_dep_wait();
    grid_dep_launch();
    const int p = blockIdx.y, tid = threadIdx.x;
    if (info[p] != 0) return;
    // the linear index of (ib, kb), kb <= ib, over the trailing blocks
    int t = (int)blockIdx.x, ib = 0;
    while (t > ib) {
        t -= ib + 1;
        ++ib;
    }
    const int kb = t;
    const int nb = min(RB, K - r0);
    const int ri = r0 + RB * (1 + ib), rk = r0 + RB * (1 + kb);
    __shared__ double Pi[RB][LD_STRIDE], Pk[RB][LD_STRIDE];
    __shared__ double D[RB * LD_STRIDE];
    double *Lp = L + (int64_t)p * K * K;
    for (int e = tid; e < RB * RB; e += blockDim.x) {
        const int a = e / RB, j = e % RB;
        Pi[a][j] = (ri + a < K && j < nb) ? Lp[(int64_t)(ri + a) * K + r0 + j] : 0.0;
        Pk[a][j] = (rk + a < K && j < nb) ? Lp[(int64_t)(rk + a) * K + r0 + j] : 0.0;
    }
    __syncthreads();
    const bool first_diag = ib == 0 && kb == 0;
    for (int e = tid; e < RB * RB; e += blockDim.x) {
        const int a = e / RB, c = e % RB;
        const int i = ri + a, k = rk + c;
        const bool in = i < K && k < K && k <= i;
        double v = 0.0;
        if (in) {
            double s = 0.0;
#pragma unroll 8
            for (int j = 0; j < RB; ++j) s = fma(Pi[a][j], Pk[c][j], s);
            v = Lp[(int64_t)i * K + k] - s;
            if (!first_diag) Lp[(int64_t)i * K + k] = v;
        }
        if (first_diag) D[a * LD_STRIDE + c] = v;
    }
    if (!first_diag) return;
    __syncthreads();
    __shared__ double r_sh;
    __shared__ int fail_sh;
    const int nb1 = min(RB, K - ri);
    const int fail = factor_diag_block(D, nb1, &r_sh, &fail_sh);
    if (fail) {
        if (tid == 0) info[p] = ri + fail;
        return;
    }
    for (int e = tid; e < RB * RB; e += blockDim.x) {
        const int i = e / RB, j = e % RB;
        if (i < nb1 && j <= i) Lp[(int64_t)(ri + i) * K + ri + j] = D[i * LD_STRIDE + j];
    }
}

// Cluster of SC blocks per (fold, chunk of up to SOLVE_MC responses): L z =
// c, then L^T b = z, by RB-row blocks.  Block c of the cluster owns the row
// blocks c, c + SC, ... and keeps their right-hand sides in shared memory.
// Each step solves one row block (forward: 0 .. nblk-1, then backward): its
// owner solves the block's triangle (a warp per response, a lane per row,
// the solved value passed by shuffle) and publishes the RB solved values;
// after the cluster barrier every block reads them from the owner's shared
// memory and, during the next step, updates its own later (forward) or
// earlier (backward) row blocks with one RB x RB tile of L each, a thread
// per (row, response).  The published buffer alternates between two slots:
// a slot is rewritten two steps later, after every block has arrived at the
// barrier that follows its reads.  A fold whose factorisation failed gets
// NaN.
constexpr int SC = 8;
constexpr int SOLVE_THREADS = 256;
constexpr int SOLVE_MC = SOLVE_THREADS / RB;   // a thread per (row, response) of a tile
constexpr size_t SOLVE_SMEM_MAX = 200 * 1024;

__host__ __device__ constexpr int solve_owned(int K) { return ((K + RB - 1) / RB + SC - 1) / SC; }

__host__ __device__ constexpr size_t solve_smem_bytes(int K, int mc) {
    return ((size_t)solve_owned(K) * RB * mc + 3 * (size_t)RB * mc + 2 * (size_t)RB * LD_STRIDE + RB) *
           sizeof(double);
}

// Cluster barrier, split: arrive releases this thread's prior writes, wait
// acquires every arrived thread's (all threads of the warp take part).
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// The owner's triangle of one row block: forward (L_bb z = v) or backward
// (L_bb^T x = v) on the block's right-hand sides Rb[r][q], copied to pub.
// S is L_bb with its columns (forward) or rows (backward) scaled by the
// reciprocal diagonal inv, so each step is one FMA: v_r -= v_i S; the
// solved values are v_r inv_r.
template <bool BACKWARD>
__device__ void solve_triangle(const double *S, const double *inv, int nb, int nm, int mc, double *Rb,
                               double *pub) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w >= nm) return;
    double v = lane < nb ? Rb[lane * mc + w] : 0.0;
    for (int s = 0; s < nb; ++s) {
        const int i = BACKWARD ? nb - 1 - s : s;
        const double vi = __shfl_sync(0xffffffffu, v, i);
        if (BACKWARD ? lane < i : (lane > i && lane < nb))
            v = fma(-vi, BACKWARD ? S[i * LD_STRIDE + lane] : S[lane * LD_STRIDE + i], v);
    }
    if (lane < nb) {
        v *= inv[lane];
        Rb[lane * mc + w] = v;
        pub[lane * mc + w] = v;
    }
}

__global__ void __cluster_dims__(SC, 1, 1) __launch_bounds__(SOLVE_THREADS)
    k_ridge_solve(int K, int M, int mc, const double *__restrict__ L, const double *__restrict__ XTY,
                  double *__restrict__ B, const int32_t *__restrict__ info) {
    grid_dep_wait();
    grid_dep_launch();
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double sm[];
    const int c = (int)cl.block_rank();
    const int p = blockIdx.y, m0 = (int)blockIdx.z * mc, nm = min(mc, M - m0);
    const int tid = threadIdx.x;
    const int nblk = (K + RB - 1) / RB;
    const int nown = c < nblk ? (nblk - 1 - c) / SC + 1 : 0;
    double *R = sm;                                        // [owned block][RB][mc]
    double *pub = R + (size_t)solve_owned(K) * RB * mc;    // [2][RB][mc]: published solved blocks
    double *zb = pub + 2 * RB * mc;                        // [RB][mc]: the block just solved
    double *T = zb + RB * mc;                              // [RB][LD_STRIDE]: a tile of L
    double *Ld = T + RB * LD_STRIDE;                       // [RB][LD_STRIDE]: a diagonal block
    double *inv = Ld + RB * LD_STRIDE;                     // [RB]: its reciprocal diagonal
    const double *Lp = L + (int64_t)p * K * K;
    const double *C = XTY + (int64_t)p * K * M;
    double *Bp = B + (int64_t)p * K * M;
    if (info[p] != 0) {   // the same for every block of the cluster
        for (int e = tid; e < nown * RB * nm; e += SOLVE_THREADS) {
            const int row = (c + SC * (e / (RB * nm))) * RB + (e % (RB * nm)) / nm;
            if (row < K) Bp[(int64_t)row * M + m0 + e % nm] = __longlong_as_double(0x7ff8000000000000LL);
        }
        return;
    }
    for (int e = tid; e < nown * RB * nm; e += SOLVE_THREADS) {
        const int j = e / (RB * nm), r = (e % (RB * nm)) / nm, q = e % nm;
        const int row = (c + SC * j) * RB + r;
        R[(j * RB + r) * mc + q] = row < K ? C[(int64_t)row * M + m0 + q] : 0.0;
    }
    const int tr = tid / SOLVE_MC, tq = tid % SOLVE_MC;   // this thread's (row, response) of a tile
    auto load_diag = [&](int r0, int nb) {
        for (int e = tid; e < RB * RB; e += SOLVE_THREADS) {
            const int i = e / RB, j = e % RB;
            Ld[i * LD_STRIDE + j] = (i < nb && j <= i) ? Lp[(int64_t)(r0 + i) * K + r0 + j] : 0.0;
        }
    };
    // the row block solved at step s: forward 0 .. nblk-1, then backward
    auto block_of = [&](int s) { return s < nblk ? s : 2 * nblk - 1 - s; };
    // Apply the values published at step sp (in zb) to the owned row blocks
    // they concern (forward: later blocks, backward: earlier ones): only
    // owned block `only` when it is >= 0, else all but owned block `skip`.
    auto apply = [&](int sp, int only, int skip) {
        const int bp = block_of(sp), r0 = bp * RB, nb = min(RB, K - r0);
        const bool bwd = sp >= nblk;
        for (int j = 0; j < nown; ++j) {
            const int bb = c + SC * j;
            if ((bwd ? bb >= bp : bb <= bp) || (only >= 0 && j != only) || j == skip) continue;
            const int s0 = bb * RB, ns = min(RB, K - s0);
            // forward: T[r][i] = L[s0 + r][r0 + i]; backward: T[r][i] = L[r0 + i][s0 + r]
            for (int e = tid; e < RB * RB; e += SOLVE_THREADS) {
                const int x = e / RB, y = e % RB;
                if (bwd) T[y * LD_STRIDE + x] = (x < nb && y < ns) ? Lp[(int64_t)(r0 + x) * K + s0 + y] : 0.0;
                else T[x * LD_STRIDE + y] = (x < ns && y < nb) ? Lp[(int64_t)(s0 + x) * K + r0 + y] : 0.0;
            }
            __syncthreads();
            if (tq < nm && tr < ns) {
                double acc = 0.0;
                for (int i = 0; i < nb; ++i) acc = fma(T[tr * LD_STRIDE + i], zb[i * mc + tq], acc);
                R[(j * RB + tr) * mc + tq] -= acc;
            }
            __syncthreads();
        }
    };
    __syncthreads();
    // Step s: the owner of block b first applies step s-1's values to block b
    // (the critical path), solves and publishes it, and only then arrives at
    // the cluster barrier; every other block arrives at once and applies
    // step s-1's values to its own blocks before it waits.  After the
    // barrier every block copies the published values.
    for (int s = 0; s < 2 * nblk; ++s) {
        const int b = block_of(s), owner = b % SC, r0 = b * RB, nb = min(RB, K - r0);
        double *slot = pub + (s & 1) * RB * mc;
        if (c == owner) {
            const int jb = b / SC;
            if (s > 0) apply(s - 1, jb, -1);
            load_diag(r0, nb);
            __syncthreads();
            if (tid < nb) inv[tid] = 1.0 / Ld[tid * LD_STRIDE + tid];
            __syncthreads();
            for (int e = tid; e < RB * RB; e += SOLVE_THREADS) {   // forward: columns, backward: rows
                const int i = e / RB, j = e % RB;
                if (j < i) Ld[i * LD_STRIDE + j] *= inv[s >= nblk ? i : j];
            }
            __syncthreads();
            double *Rb = R + (size_t)jb * RB * mc;
            if (s >= nblk) solve_triangle<true>(Ld, inv, nb, nm, mc, Rb, slot);
            else solve_triangle<false>(Ld, inv, nb, nm, mc, Rb, slot);
            cluster_arrive();
            if (s > 0) apply(s - 1, -1, jb);
        } else {
            cluster_arrive();
            if (s > 0) apply(s - 1, -1, -1);
        }
        cluster_wait();
        __syncthreads();   // every thread is done with zb
        const double *src = cl.map_shared_rank(slot, owner);
        for (int e = tid; e < nb * nm; e += SOLVE_THREADS) zb[(e / nm) * mc + e % nm] = src[(e / nm) * mc + e % nm];
        __syncthreads();
    }
    for (int e = tid; e < nown * RB * nm; e += SOLVE_THREADS) {
        const int j = e / (RB * nm), r = (e % (RB * nm)) / nm, q = e % nm;
        const int row = (c + SC * j) * RB + r;
        if (row < K) Bp[(int64_t)row * M + m0 + q] = R[(j * RB + r) * mc + q];
    }
    cluster_arrive();   // no block leaves while another may still read its published values
    cluster_wait();
}

__host__ __device__ constexpr size_t press_smem_bytes(int K, int mc) {
    return ((size_t)mc * K + K + 2 * (size_t)mc + (size_t)PRESS_WARPS * mc) * sizeof(double);
}

// Block per contiguous range of the fold-sorted rows (the N rows split evenly
// over the grid).  For each fold the range meets and each chunk of up to mc
// responses, the block stages in shared memory the model as it applies to
// the raw X values, B~[q][k] = B_p[k][m0 + q] / ([sX] ? std_k : 1), the
// centring vector ([cX] ? mean_k : 0) and Y's scale and shift; a warp per
// row then forms x~ B~ (lanes over k, coalesced reads of the row), maps it
// back to Y's units and sums the squared residuals.  One atomicAdd per
// (block, fold, response).  Dividing B rather than each x by std changes
// only the rounding, by about one unit in the last place per term.
template <typename T>
__global__ void __launch_bounds__(PRESS_THREADS)
    k_ridge_press(const __grid_constant__ PlanView pl, const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y,
                  int64_t ldy, int flags, const double *__restrict__ mean, const double *__restrict__ std,
                  const double *__restrict__ B, int mc, double *__restrict__ press) {
    grid_dep_wait();
    grid_dep_launch();
    extern __shared__ double sm[];
    const int K = pl.K, M = pl.M, KM = K + M;
    double *Bs = sm;                       // [mc][K]
    double *mus = Bs + (size_t)mc * K;     // [K]
    double *ysd = mus + K;                 // [mc]
    double *ymu = ysd + mc;                // [mc]
    double *red = ymu + mc;                // [PRESS_WARPS][mc]
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t R0 = pl.N * (int64_t)blockIdx.x / gridDim.x;
    const int64_t R1 = pl.N * (int64_t)(blockIdx.x + 1) / gridDim.x;
    if (R0 >= R1) return;
    const bool cx = flags & CV_CENTER_X, sx = flags & CV_SCALE_X;
    const bool cy = flags & CV_CENTER_Y, sy = flags & CV_SCALE_Y;
    int lo = 0, hi = pl.P - 1;   // fold of R0: the last p with offs[p] <= R0
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (pl.offs[mid] <= R0) lo = mid;
        else hi = mid - 1;
    }
    int p = lo;
    for (int64_t a = R0; a < R1;) {
        while (pl.offs[p + 1] <= a) ++p;
        const int64_t b = min(R1, pl.offs[p + 1]);
        const double *mu = mean + (int64_t)p * KM, *sd = std + (int64_t)p * KM;
        const double *Bp = B + (int64_t)p * K * M;
        for (int m0 = 0; m0 < M; m0 += mc) {
            const int nm = min(mc, M - m0);
            __syncthreads();   // the previous pass is done with the staged values
            for (int64_t e = tid; e < (int64_t)K * nm; e += PRESS_THREADS) {
                const int k = (int)(e / nm), q = (int)(e % nm);
                const double bv = Bp[(int64_t)k * M + m0 + q];
                Bs[(int64_t)q * K + k] = sx ? bv / sd[k] : bv;
            }
            for (int k = tid; k < K; k += PRESS_THREADS) mus[k] = cx ? mu[k] : 0.0;
            if (tid < nm) {
                ysd[tid] = sy ? sd[K + m0 + tid] : 1.0;
                ymu[tid] = cy ? mu[K + m0 + tid] : 0.0;
            }
            __syncthreads();
            double acc[PRESS_MC];
#pragma unroll
            for (int q = 0; q < PRESS_MC; ++q) acc[q] = 0.0;
            for (int64_t r = a + w; r < b; r += PRESS_WARPS) {
                const int64_t n = pl.perm[r];
                const T *xr = X + n * ldx;
                double pred[PRESS_MC];
#pragma unroll
                for (int q = 0; q < PRESS_MC; ++q) pred[q] = 0.0;
                for (int k = lane; k < K; k += 32) {
                    const double xt = (double)xr[k] - mus[k];
#pragma unroll
                    for (int q = 0; q < PRESS_MC; ++q)
                        if (q < nm) pred[q] = fma(xt, Bs[(int64_t)q * K + k], pred[q]);
                }
#pragma unroll
                for (int q = 0; q < PRESS_MC; ++q) {
                    if (q < nm) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) pred[q] += __shfl_xor_sync(0xffffffffu, pred[q], o);
                        const double res = (double)Y[n * ldy + m0 + q] - (pred[q] * ysd[q] + ymu[q]);
                        acc[q] = fma(res, res, acc[q]);
                    }
                }
            }
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < PRESS_MC; ++q)
                    if (q < nm) red[w * mc + q] = acc[q];
            __syncthreads();
            if (tid < nm) {
                double t = 0.0;
                for (int ww = 0; ww < PRESS_WARPS; ++ww) t += red[ww * mc + tid];
                atomicAdd(press + (int64_t)p * M + m0 + tid, t);
            }
        }
        a = b;
    }
}

}  // namespace
}  // namespace cvx

extern "C" {

cv_status cv_ridge(int32_t P, int32_t K, int32_t M, const double *XTX, const double *XTY, double lambda, double *L,
                   double *B, int32_t *info, void *stream) {
    if (P < 1 || K < 1 || M < 0 || !XTX || !L || !info || (M > 0 && (!XTY || !B)) || !isfinite(lambda))
        return CV_ERR_INVALID_ARG;
    // folds are a grid dimension; one response's right-hand side must fit in shared memory
    if (P > 65535 || (M > 0 && cvx::solve_smem_bytes(K, 1) > cvx::SOLVE_SMEM_MAX)) return CV_ERR_UNSUPPORTED;
    using namespace cvx;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t KK = (int64_t)K * K;
    const unsigned init_blocks = (unsigned)std::min<int64_t>(1024, (KK + 255) / 256);
    cudaError_t e = launch_pdl(k_ridge_init, dim3(init_blocks, (unsigned)P), dim3(256), 0, st, (int)K, XTX, lambda, L,
                               info);
    if (e == cudaSuccess) e = launch_pdl(k_ridge_potrf, dim3((unsigned)P), dim3(256), 0, st, (int)K, L, info);
    const int nblk = (K + RB - 1) / RB;
    for (int b = 0; b + 1 < nblk && e == cudaSuccess; ++b) {
        const int r0 = b * RB, T = nblk - b - 1;   // blocks below the diagonal block
        e = launch_pdl(k_ridge_trsm, dim3((unsigned)T, (unsigned)P), dim3(TRSM_THREADS), 0, st, (int)K, r0, L,
                       (const int32_t *)info);
        if (e == cudaSuccess)
            e = launch_pdl(k_ridge_update, dim3((unsigned)(T * (T + 1) / 2), (unsigned)P), dim3(256), 0, st, (int)K,
                           r0, L, info);
    }
    if (e == cudaSuccess && M > 0) {
        int mc = std::min(SOLVE_MC, (int)M);
        while (mc > 1 && solve_smem_bytes(K, mc) > SOLVE_SMEM_MAX) --mc;
        if ((M + mc - 1) / mc > 65535) return CV_ERR_UNSUPPORTED;   // response chunks are a grid dimension
        const size_t smem = solve_smem_bytes(K, mc);
        e = cudaFuncSetAttribute(k_ridge_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = launch_pdl(k_ridge_solve, dim3(SC, (unsigned)P, (unsigned)((M + mc - 1) / mc)), dim3(SOLVE_THREADS),
                           smem, st, (int)K, (int)M, mc, (const double *)L, XTY, B, (const int32_t *)info);
    }
    return e == cudaSuccess ? CV_OK : CV_ERR_CUDA;
}

cv_status cv_ridge_press(cv_plan_t plan, const void *X, int64_t ldx, const void *Y, int64_t ldy, int flags,
                         const double *mean, const double *std, const double *B, double *press, void *stream) {
    if (!plan || !X || !Y || !mean || !std || !B || !press) return CV_ERR_INVALID_ARG;
    if (plan->sharded) return CV_ERR_UNSUPPORTED;   // works on plans of every fold
    const cvx::PlanView &v = plan->v;
    if (v.M < 1 || ldx < v.K || ldy < v.M || flags < 0 || flags > 15) return CV_ERR_INVALID_ARG;
    using namespace cvx;
    int mc = std::min(PRESS_MC, v.M);
    while (mc > 1 && press_smem_bytes(v.K, mc) > PRESS_SMEM_TARGET) --mc;
    const size_t smem = press_smem_bytes(v.K, mc);
    if (smem > PRESS_SMEM_MAX) return CV_ERR_UNSUPPORTED;   // one response's model must fit in shared memory
    cudaStream_t st = (cudaStream_t)stream;
    const bool f32 = plan->in_dtype == CV_F32;
    const void *kern = f32 ? (const void *)k_ridge_press<float> : (const void *)k_ridge_press<double>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 1;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PRESS_THREADS, smem);
    // blocks of at least 64 rows, at most as many as are resident at once
    const int64_t blocks = std::max<int64_t>(
        1, std::min<int64_t>((v.N + 63) / 64, (int64_t)plan->num_sms * std::max(1, per_sm)));
    if (e == cudaSuccess) e = cudaMemsetAsync(press, 0, sizeof(double) * (size_t)v.P * v.M, st);
    if (e == cudaSuccess) {
        if (f32)
            e = launch_pdl(k_ridge_press<float>, dim3((unsigned)blocks), dim3(PRESS_THREADS), smem, st, v,
                           (const float *)X, ldx, (const float *)Y, ldy, flags, mean, std, B, mc, press);
        else
            e = launch_pdl(k_ridge_press<double>, dim3((unsigned)blocks), dim3(PRESS_THREADS), smem, st, v,
                           (const double *)X, ldx, (const double *)Y, ldy, flags, mean, std, B, mc, press);
    }
    return e == cudaSuccess ? CV_OK : CV_ERR_CUDA;
}

}  // extern "C"
