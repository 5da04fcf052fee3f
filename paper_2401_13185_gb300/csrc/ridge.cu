// ridge.cu -- per-fold ridge regression / OLS on the products, and the
// models' squared error on each validation partition.
//
// The paper names ridge regression and OLS through the normal equations as
// consumers of X^T X and X^T Y, and cross-validation as fitting on each
// training partition and evaluating on its validation partition (Section 1).
//
//   cv_ridge        For each fold p, B_p = (XTX_p + lambda I)^-1 XTY_p by the
//                   Cholesky factorisation XTX_p + lambda I = L L^T in FP64,
//                   then forward and back substitution.  One block per fold.
//   cv_ridge_press  press[p][m] = sum over the validation rows n of fold p of
//                   (y_nm - y^_nm)^2.  Each validation row is preprocessed
//                   with its fold's TRAINING statistics (x~ = (x - [cX] mean)
//                   / ([sX] ? std : 1)), predicted in that space (x~ B_p) and
//                   mapped back to Y's units (times [sY] std, plus [cY] mean).
//
// All arithmetic is FP64; the work is small next to the products (K^3 / 3
// per fold for the factorisation, N K M for the predictions).
#include <math.h>

#include "cvx_internal.cuh"

namespace cvx {
namespace {

constexpr int RIDGE_THREADS = 256;
constexpr int PRESS_THREADS = 256;
constexpr int PRESS_ROWS_PER_WARP = 64;
constexpr int PRESS_RCH = 8;   // responses per pass over a row

// Sum over the block; the result is valid in thread 0 only.  The caller
// synchronises the block before `red` is written again.
__device__ __forceinline__ double block_sum_t0(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < RIDGE_THREADS / 32; ++w) s += red[w];
    return s;
}

// Block per fold.  Column j of L: the pivot d = sqrt(a_jj + lambda -
// sum_{k<j} L[j][k]^2), then L[i][j] = (a_ij - sum_{k<j} L[i][k] L[j][k]) / d
// for i > j, one thread per row i.  L is kept column-major (Lc[k K + i] =
// L[i][k]) so that the threads of one column read consecutive addresses.
// Only the lower triangle of XTX_p is read.  Then B_p = XTY_p, L z = B_p
// (once z_i is known its multiple of column i of L leaves the rows below) and
// L^T b = z (likewise upwards).
__global__ void __launch_bounds__(RIDGE_THREADS)
    k_ridge(int K, int M, const double *__restrict__ XTX, const double *__restrict__ XTY, double lambda,
            double *__restrict__ Lws, double *__restrict__ B, int32_t *__restrict__ info) {
    grid_dep_wait();
    grid_dep_launch();
    const int p = blockIdx.x, tid = threadIdx.x;
    const double *A = XTX + (int64_t)p * K * K;
    double *Lc = Lws + (int64_t)p * K * K;
    double *Bp = B + (int64_t)p * K * M;
    __shared__ double red[RIDGE_THREADS / 32];
    __shared__ double piv;
    __shared__ int fail;
    if (tid == 0) fail = 0;
    for (int j = 0; j < K; ++j) {
        double part = 0.0;
        for (int k = tid; k < j; k += RIDGE_THREADS) {
            const double l = Lc[(int64_t)k * K + j];
            part += l * l;
        }
        const double s = block_sum_t0(part, red);
        if (tid == 0) {
            const double d2 = A[(int64_t)j * K + j] + lambda - s;
            if (d2 > 0.0) {
                piv = sqrt(d2);
                Lc[(int64_t)j * K + j] = piv;
            } else {
                fail = j + 1;
            }
        }
        __syncthreads();
        if (fail) break;
        const double d = piv;
        for (int i = j + 1 + tid; i < K; i += RIDGE_THREADS) {
            double t = A[(int64_t)i * K + j];
            for (int k = 0; k < j; ++k) t -= Lc[(int64_t)k * K + i] * Lc[(int64_t)k * K + j];
            Lc[(int64_t)j * K + i] = t / d;
        }
        __syncthreads();
    }
    if (fail) {
        if (tid == 0) info[p] = fail;
        for (int64_t e = tid; e < (int64_t)K * M; e += RIDGE_THREADS) Bp[e] = nan("");
        return;
    }
    if (tid == 0) info[p] = 0;
    const double *C = XTY + (int64_t)p * K * M;
    for (int64_t e = tid; e < (int64_t)K * M; e += RIDGE_THREADS) Bp[e] = C[e];
    __syncthreads();
    for (int i = 0; i < K; ++i) {   // L z = c
        const double lii = Lc[(int64_t)i * K + i];
        for (int m = tid; m < M; m += RIDGE_THREADS) Bp[(int64_t)i * M + m] /= lii;
        __syncthreads();
        const int64_t below = (int64_t)(K - 1 - i) * M;
        for (int64_t e = tid; e < below; e += RIDGE_THREADS) {
            const int k = i + 1 + (int)(e / M), m = (int)(e % M);
            Bp[(int64_t)k * M + m] -= Lc[(int64_t)i * K + k] * Bp[(int64_t)i * M + m];
        }
        __syncthreads();
    }
    for (int i = K - 1; i >= 0; --i) {   // L^T b = z
        const double lii = Lc[(int64_t)i * K + i];
        for (int m = tid; m < M; m += RIDGE_THREADS) Bp[(int64_t)i * M + m] /= lii;
        __syncthreads();
        const int64_t above = (int64_t)i * M;
        for (int64_t e = tid; e < above; e += RIDGE_THREADS) {
            const int k = (int)(e / M), m = (int)(e % M);
            Bp[(int64_t)k * M + m] -= Lc[(int64_t)k * K + i] * Bp[(int64_t)i * M + m];
        }
        __syncthreads();
    }
}

// Warp per run of PRESS_ROWS_PER_WARP rows in fold-sorted order.  Lanes split
// a row's K columns: each lane preprocesses its columns with the fold's
// training statistics and accumulates their share of PRESS_RCH predictions;
// a butterfly reduction gives every lane the predictions; the squared
// residuals are summed per response while the run stays in one fold and
// added to press (one atomicAdd per response) when it leaves the fold.
template <typename T>
__global__ void __launch_bounds__(PRESS_THREADS)
    k_ridge_press(const __grid_constant__ PlanView pl, const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y,
                  int64_t ldy, int flags, const double *__restrict__ mean, const double *__restrict__ std,
                  const double *__restrict__ B, double *__restrict__ press) {
    grid_dep_wait();
    grid_dep_launch();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * PRESS_THREADS + threadIdx.x) >> 5;
    const int64_t r0 = warp * PRESS_ROWS_PER_WARP;
    if (r0 >= pl.N) return;
    const int64_t r1 = min(pl.N, r0 + (int64_t)PRESS_ROWS_PER_WARP);
    const int K = pl.K, M = pl.M, KM = K + M;
    const bool cx = flags & CV_CENTER_X, sx = flags & CV_SCALE_X;
    const bool cy = flags & CV_CENTER_Y, sy = flags & CV_SCALE_Y;
    // fold of r0: the last p with offs[p] <= r0
    int lo = 0, hi = pl.P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (pl.offs[mid] <= r0) lo = mid;
        else hi = mid - 1;
    }
    const int p_first = lo;
    for (int m0 = 0; m0 < M; m0 += PRESS_RCH) {
        int p = p_first;
        int64_t p_end = pl.offs[p + 1];
        double acc[PRESS_RCH];
#pragma unroll
        for (int q = 0; q < PRESS_RCH; ++q) acc[q] = 0.0;
        auto flush = [&]() {
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < PRESS_RCH; ++q)
                    if (m0 + q < M) atomicAdd(press + (int64_t)p * M + m0 + q, acc[q]);
            }
#pragma unroll
            for (int q = 0; q < PRESS_RCH; ++q) acc[q] = 0.0;
        };
        for (int64_t r = r0; r < r1; ++r) {
            while (r >= p_end) {
                flush();
                ++p;
                p_end = pl.offs[p + 1];
            }
            const int64_t n = pl.perm[r];
            const double *mu = mean + (int64_t)p * KM, *sd = std + (int64_t)p * KM;
            const double *Bp = B + (int64_t)p * K * M + m0;
            double pred[PRESS_RCH];
#pragma unroll
            for (int q = 0; q < PRESS_RCH; ++q) pred[q] = 0.0;
            for (int k = lane; k < K; k += 32) {
                double xt = (double)X[n * ldx + k];
                if (cx) xt -= mu[k];
                if (sx) xt /= sd[k];
#pragma unroll
                for (int q = 0; q < PRESS_RCH; ++q)
                    if (m0 + q < M) pred[q] += xt * Bp[(int64_t)k * M + q];
            }
#pragma unroll
            for (int q = 0; q < PRESS_RCH; ++q) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) pred[q] += __shfl_xor_sync(0xffffffffu, pred[q], o);
            }
#pragma unroll
            for (int q = 0; q < PRESS_RCH; ++q) {
                const int m = m0 + q;
                if (m < M) {
                    double yhat = pred[q];
                    if (sy) yhat *= sd[K + m];
                    if (cy) yhat += mu[K + m];
                    const double res = (double)Y[n * ldy + m] - yhat;
                    acc[q] += res * res;
                }
            }
        }
        flush();
    }
}

}  // namespace
}  // namespace cvx

extern "C" {

cv_status cv_ridge(int32_t P, int32_t K, int32_t M, const double *XTX, const double *XTY, double lambda, double *L,
                   double *B, int32_t *info, void *stream) {
    if (P < 1 || K < 1 || M < 0 || !XTX || !L || !info || (M > 0 && (!XTY || !B)) || !isfinite(lambda))
        return CV_ERR_INVALID_ARG;
    const cudaError_t e = cvx::launch_pdl(cvx::k_ridge, dim3((unsigned)P), dim3(cvx::RIDGE_THREADS), 0,
                                          (cudaStream_t)stream, (int)K, (int)M, XTX, XTY, lambda, L, B, info);
    return e == cudaSuccess ? CV_OK : CV_ERR_CUDA;
}

cv_status cv_ridge_press(cv_plan_t plan, const void *X, int64_t ldx, const void *Y, int64_t ldy, int flags,
                         const double *mean, const double *std, const double *B, double *press, void *stream) {
    if (!plan || !X || !Y || !mean || !std || !B || !press) return CV_ERR_INVALID_ARG;
    if (plan->sharded) return CV_ERR_UNSUPPORTED;   // works on plans of every fold
    const cvx::PlanView &v = plan->v;
    if (v.M < 1 || ldx < v.K || ldy < v.M || flags < 0 || flags > 15) return CV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(press, 0, sizeof(double) * (size_t)v.P * v.M, st);
    const int64_t warps = (v.N + cvx::PRESS_ROWS_PER_WARP - 1) / cvx::PRESS_ROWS_PER_WARP;
    const unsigned blocks = (unsigned)((warps * 32 + cvx::PRESS_THREADS - 1) / cvx::PRESS_THREADS);
    if (e == cudaSuccess) {
        if (plan->in_dtype == CV_F32)
            e = cvx::launch_pdl(cvx::k_ridge_press<float>, dim3(blocks), dim3(cvx::PRESS_THREADS), 0, st, v,
                                (const float *)X, ldx, (const float *)Y, ldy, flags, mean, std, B, press);
        else
            e = cvx::launch_pdl(cvx::k_ridge_press<double>, dim3(blocks), dim3(cvx::PRESS_THREADS), 0, st, v,
                                (const double *)X, ldx, (const double *)Y, ldy, flags, mean, std, B, press);
    }
    return e == cudaSuccess ? CV_OK : CV_ERR_CUDA;
}

}  // extern "C"
