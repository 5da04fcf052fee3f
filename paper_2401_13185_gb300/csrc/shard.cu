// shard.cu -- fold sharding over several GPUs: cv_plan_exchange_size,
// cv_products_partial and cv_finalize_total.
//
// Lemma 2: the Gram over all rows is the sum over the folds of their
// validation Grams, so the total H_R = W^T W that every fold's training
// products subtract from (Lemma 3) is the sum of the shards' partial totals,
// each over the rows of the folds one GPU owns.  A shard's plan cuts
// segments only from its own folds (with the operand scale of the whole
// problem, so the shards' units agree); cv_products_partial contracts them,
// reduces its fold sums and its partial total, and copies the total to the
// caller's exchange buffers.  After the caller has summed the buffers over
// the shards, cv_finalize_total puts the total back and runs the statistics
// and the epilogue of the shard's folds.  The exchange is the upper block
// triangle of H in the contraction's units, 128 x 128 tiles: on the split
// path the exact int64 sums of hi * hi and the cross terms widened to FP64
// (so that the sum over the shards adds no FP32 rounding), on the FP64 path
// the FP64 sums.
#include "cvx_internal.cuh"

namespace cvx {
namespace {

__global__ void __launch_bounds__(256) k_export_total(PlanView pl, long long *__restrict__ ex_int,
                                                      double *__restrict__ ex_real) {
    grid_dep_wait();
    grid_dep_launch();
    const int64_t nt = (int64_t)pl.ntiles * TILE_ELEMS;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    if (pl.split) {
        const long long *hi = reinterpret_cast<const long long *>(pl.gtot);
        const float *lo = reinterpret_cast<const float *>(hi + nt);
        ex_int[i] = hi[i];
        ex_real[i] = (double)lo[i];
    } else {
        ex_real[i] = reinterpret_cast<const double *>(pl.gtot)[i];
    }
}

__global__ void __launch_bounds__(256) k_import_total(PlanView pl, const long long *__restrict__ ex_int,
                                                      const double *__restrict__ ex_real) {
    grid_dep_wait();
    grid_dep_launch();
    const int64_t nt = (int64_t)pl.ntiles * TILE_ELEMS;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    if (pl.split) {
        long long *hi = reinterpret_cast<long long *>(pl.gtot);
        float *lo = reinterpret_cast<float *>(hi + nt);
        hi[i] = ex_int[i];
        lo[i] = (float)ex_real[i];
    } else {
        reinterpret_cast<double *>(pl.gtot)[i] = ex_real[i];
    }
}

}  // namespace

cudaError_t export_total(const cv_plan_s *pl, long long *ex_int, double *ex_real, cudaStream_t st) {
    const int64_t nt = (int64_t)pl->v.ntiles * TILE_ELEMS;
    ++pl->launches;
    return launch_pdl(k_export_total, dim3((unsigned)((nt + 255) / 256)), dim3(256), 0, st, pl->v, ex_int, ex_real);
}

cudaError_t import_total(const cv_plan_s *pl, const long long *ex_int, const double *ex_real, cudaStream_t st) {
    const int64_t nt = (int64_t)pl->v.ntiles * TILE_ELEMS;
    ++pl->launches;
    return launch_pdl(k_import_total, dim3((unsigned)((nt + 255) / 256)), dim3(256), 0, st, pl->v, ex_int, ex_real);
}

}  // namespace cvx

using namespace cvx;

namespace {

// Make the plan's device current for the call; restores the caller's on exit.
struct DeviceScope {
    int prev = -1;
    int dev = -1;
    bool ok = false;
    explicit DeviceScope(int d) : dev(d) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope() {
        if (ok && prev != dev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

cv_status cv_plan_exchange_size(cv_plan_t pl, int64_t *n_int, int64_t *n_real) {
    if (!pl || !n_int || !n_real) return CV_ERR_INVALID_ARG;
    const int64_t nt = (int64_t)pl->v.ntiles * TILE_ELEMS;
    *n_int = pl->v.split ? nt : 0;
    *n_real = nt;
    return CV_OK;
}

cv_status cv_products_partial(cv_plan_t pl, const void *X, int64_t ldx, const void *Y, int64_t ldy, int64_t *ex_int,
                              double *ex_real, void *stream) {
    if (!pl || !pl->sharded || !ex_real || (pl->v.split && !ex_int)) return CV_ERR_INVALID_ARG;
    const cv_status chk = products_arg_status(pl, X, ldx, Y, ldy, 0, 0);   // the inputs only
    if (chk != CV_OK) return chk;
    DeviceScope ds(pl->device);
    if (!ds.ok) return CV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const bool split = pl->v.split != 0;
    cudaError_t e = shift_estimate(pl, X, ldx, Y, ldy, split, st);
    if (e == cudaSuccess && split) e = convert_split(pl, X, ldx, Y, ldy, st);
    if (e == cudaSuccess) e = split ? gram_tc(pl, st) : gram_f64(pl, X, ldx, Y, ldy, st);
    if (e == cudaSuccess) e = fold_sums(pl, st);
    if (e == cudaSuccess) e = export_total(pl, reinterpret_cast<long long *>(ex_int), ex_real, st);
    if (e == cudaSuccess) pl->has_partial = true;
    return status_of(e);
}

cv_status cv_finalize_total(cv_plan_t pl, const int64_t *ex_int, const double *ex_real, int flags, int ddof,
                            void *XTX, void *XTY, double *mean_out, double *std_out, void *stream) {
    if (!pl || !pl->sharded || !pl->has_partial || !ex_real || (pl->v.split && !ex_int)) return CV_ERR_INVALID_ARG;
    const cv_status chk = flags_arg_status(pl, flags, ddof);
    if (chk != CV_OK) return chk;
    DeviceScope ds(pl->device);
    if (!ds.ok) return CV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = import_total(pl, reinterpret_cast<const long long *>(ex_int), ex_real, st);
    if (e == cudaSuccess) e = fold_stats(pl, flags, ddof, mean_out, std_out, st);
    if (e == cudaSuccess && (XTX || XTY)) e = epilogue(pl, flags, XTX, XTY, st);
    if (e == cudaSuccess) pl->has_sums = true;
    return status_of(e);
}

}  // extern "C"
