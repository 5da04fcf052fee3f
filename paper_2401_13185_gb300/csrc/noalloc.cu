// noalloc.cu -- cv_products_f64_static: the FP64 fold products for small
// problems without allocating any memory.
//
// Some callers cannot allocate device memory: code that runs inside a process
// whose GPU memory is owned by another framework's allocator under a fixed
// budget, or a latency-critical loop where cudaMalloc (which can synchronize
// the device and can fail under memory pressure) is not acceptable.  This
// entry point serves them.  It runs the same kernels as the plan-based
// CV_PREC_FP64 path (fold count and stable fold sort, shift estimate, FP64
// Gram, fold sums, statistics, epilogue), but every scratch buffer those
// kernels need is carved from one file-scope device array,
// g_cv_static_scratch, that exists once on every GPU that loads the library
// and lives until the process exits.  Host-side bookkeeping uses fixed-size
// arrays on the stack.
//
// Limits (checked on entry; larger problems return CV_ERR_UNSUPPORTED):
// N <= 32768 rows, K + M + 1 <= 128, 2 <= P <= 16 folds.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "cvx_internal.cuh"

using namespace cvx;

namespace {

constexpr int64_t SA_MAX_N = 32768;
constexpr int32_t SA_MAX_D = TILE;   // one tile of H
constexpr int32_t SA_MAX_P = 16;
constexpr int32_t SA_MAX_SEGS = 64;
constexpr int SA_MAX_DEVICES = 64;

constexpr size_t sa_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t SA_SORT_TMP = fold_sort_tmp_bytes_for(SA_MAX_N);
// region offsets inside the scratch array (each 256-byte aligned)
constexpr size_t SA_PERM = 0;
constexpr size_t SA_TMP = SA_PERM + sa_align(sizeof(int32_t) * SA_MAX_N);
constexpr size_t SA_COUNTS = SA_TMP + sa_align(SA_SORT_TMP);
constexpr size_t SA_OFFS = SA_COUNTS + sa_align(sizeof(unsigned long long) * SA_MAX_P + sizeof(int));
constexpr size_t SA_SEGS = SA_OFFS + sa_align(sizeof(int64_t) * (SA_MAX_P + 1));
constexpr size_t SA_FSEG = SA_SEGS + sa_align(sizeof(Segment) * SA_MAX_SEGS);
constexpr size_t SA_TILES = SA_FSEG + sa_align(sizeof(int32_t) * (SA_MAX_P + 1));
constexpr size_t SA_PART = SA_TILES + sa_align(sizeof(TileCoord));
constexpr size_t SA_GFOLD = SA_PART + sa_align(sizeof(double) * SA_MAX_SEGS * TILE_ELEMS);
constexpr size_t SA_GTOT = SA_GFOLD + sa_align(sizeof(double) * SA_MAX_P * TILE_ELEMS);
constexpr size_t SA_SHIFT = SA_GTOT + sa_align(sizeof(double) * TILE_ELEMS);
constexpr size_t SA_ISC = SA_SHIFT + sa_align(sizeof(double) * SA_MAX_D);
constexpr size_t SA_SHF = SA_ISC + sa_align(sizeof(double) * SA_MAX_D);
constexpr size_t SA_SCF = SA_SHF + sa_align(sizeof(float) * SA_MAX_D);
constexpr size_t SA_STATS = SA_SCF + sa_align(sizeof(float) * SA_MAX_D);
constexpr size_t SA_ERR = SA_STATS + sa_align(sizeof(double) * 4 * SA_MAX_P * SA_MAX_D);
constexpr size_t SA_BYTES = SA_ERR + 256;   // about 11 MB

// The scratch every call shares.  Host code must not use this name as an
// address: it only stands for the symbol; the device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_cv_static_scratch[SA_BYTES];

std::mutex g_sa_mutex;
void *g_sa_ptr[SA_MAX_DEVICES];

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t static_scratch(int dev, void **out) {
    std::lock_guard<std::mutex> lock(g_sa_mutex);
    if (!g_sa_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_cv_static_scratch);
        if (e != cudaSuccess) return e;
        g_sa_ptr[dev] = p;
    }
    *out = g_sa_ptr[dev];
    return cudaSuccess;
}

cv_status to_status(cudaError_t e) { return e == cudaSuccess ? CV_OK : CV_ERR_CUDA; }

}  // namespace

extern "C" cv_status cv_products_f64_static(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *fold_ids,
                                            const void *X, int64_t ldx, const void *Y, int64_t ldy,
                                            cv_dtype in_dtype, cv_dtype out_dtype, int flags, int ddof, void *XTX,
                                            void *XTY, double *mean_out, double *std_out, void *stream) {
    if (N < 2 || K < 1 || M < 0 || P < 2 || (int64_t)P > N || !fold_ids || !X) return CV_ERR_INVALID_ARG;
    if (M > 0 && (!Y || ldy < M)) return CV_ERR_INVALID_ARG;
    if (ldx < K || flags < 0 || flags > 15 || ddof < 0 || ddof > 1) return CV_ERR_INVALID_ARG;
    if ((in_dtype != CV_F32 && in_dtype != CV_F64) || (out_dtype != CV_F32 && out_dtype != CV_F64))
        return CV_ERR_INVALID_ARG;
    if (N > SA_MAX_N || (int64_t)K + M + 1 > SA_MAX_D || P > SA_MAX_P) return CV_ERR_UNSUPPORTED;

    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return CV_ERR_CUDA;
    if (dev < 0 || dev >= SA_MAX_DEVICES) return CV_ERR_UNSUPPORTED;
    void *scratch = nullptr;
    if ((e = static_scratch(dev, &scratch)) != cudaSuccess) return CV_ERR_CUDA;
    char *base = (char *)scratch;

    // The plan view over the static scratch (std::vector members stay empty).
    cv_plan_s pl{};
    pl.opts = cv_plan_options{CV_STRATEGY_AUTO, 0};
    pl.in_dtype = in_dtype;
    pl.out_dtype = out_dtype;
    pl.prec = CV_PREC_FP64;
    pl.device = dev;
    pl.d_block = nullptr;
    pl.ws_bytes = SA_BYTES;
    pl.ypack = nullptr;
    pl.ypack_width = 0;
    pl.profiling = false;
    pl.prof_calls = 0;
    pl.launches = 0;
    pl.has_sums = false;
    if (cudaDeviceGetAttribute(&pl.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CV_ERR_CUDA;
    PlanView &v = pl.v;
    memset(&v, 0, sizeof(v));
    v.N = N;
    v.K = K;
    v.M = M;
    v.P = P;
    v.D = K + M + 1;
    v.nb = 1;
    v.ntiles = 1;
    v.nlast = TILE;
    v.p_lo = 0;        // every fold, full X^T X layout
    v.p_hi = P;
    v.packed = 0;
    v.wait_ns = 1000000000ull;
    v.split = 0;
    v.perm = (int32_t *)(base + SA_PERM);
    v.offs = (int64_t *)(base + SA_OFFS);
    v.segs = (Segment *)(base + SA_SEGS);
    v.fold_seg = (int32_t *)(base + SA_FSEG);
    v.tiles = (TileCoord *)(base + SA_TILES);
    v.partials = (double *)(base + SA_PART);
    v.gfold = (void *)(base + SA_GFOLD);
    v.gtot = (void *)(base + SA_GTOT);
    v.sp.shift = (double *)(base + SA_SHIFT);
    v.sp.inv_scale = (double *)(base + SA_ISC);
    v.sp.shift_f = (float *)(base + SA_SHF);
    v.sp.scale_f = (float *)(base + SA_SCF);
    v.stats = (double *)(base + SA_STATS);
    v.err = (int *)(base + SA_ERR);

    // Algorithm 1 on the device: validate and count (the counts start at zero:
    // the array keeps the previous call's contents).
    unsigned long long *d_cnt = (unsigned long long *)(base + SA_COUNTS);
    int *d_bad = (int *)(d_cnt + P);
    e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * P + sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.err, 0, sizeof(int) * 4, st);
    if (e == cudaSuccess) e = fold_count(fold_ids, N, P, d_cnt, d_bad, st);
    unsigned long long counts[SA_MAX_P];
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, d_cnt, sizeof(unsigned long long) * P, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return CV_ERR_CUDA;
    if (bad) return CV_ERR_FOLD_RANGE;
    int64_t offs[SA_MAX_P + 1];
    offs[0] = 0;
    for (int p = 0; p < P; ++p) {
        if (counts[p] == 0) return CV_ERR_EMPTY_FOLD;
        offs[p + 1] = offs[p] + (int64_t)counts[p];
    }
    if (flags & (CV_SCALE_X | CV_SCALE_Y))
        for (int p = 0; p < P; ++p)
            if (N - (offs[p + 1] - offs[p]) - ddof < 1) return CV_ERR_NOT_SCALABLE;

    // Segments: at most SA_MAX_SEGS, never straddling a fold.
    const int64_t rows_per_seg = std::max<int64_t>(256, (N + (SA_MAX_SEGS - P) - 1) / (SA_MAX_SEGS - P));
    Segment segs[SA_MAX_SEGS];
    int32_t fold_seg[SA_MAX_P + 1];
    int ns = 0;
    for (int p = 0; p < P; ++p) {
        fold_seg[p] = ns;
        const int64_t nv = offs[p + 1] - offs[p];
        const int64_t k = (nv + rows_per_seg - 1) / rows_per_seg;
        for (int64_t q = 0; q < k; ++q) {
            segs[ns].begin = (int32_t)(offs[p] + nv * q / k);
            segs[ns].end = (int32_t)(offs[p] + nv * (q + 1) / k);
            segs[ns].fold = p;
            segs[ns].pad = 0;
            ++ns;
        }
    }
    fold_seg[P] = ns;
    v.nsegs = ns;
    const TileCoord tile{0, 0};
    v.nsample = (int32_t)std::min<int64_t>(N, SHIFT_SAMPLE);

    e = fold_sort(fold_ids, N, P, v.perm, base + SA_TMP, SA_SORT_TMP, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v.offs, offs, sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v.segs, segs, sizeof(Segment) * ns, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(v.fold_seg, fold_seg, sizeof(int32_t) * (P + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v.tiles, &tile, sizeof(TileCoord), cudaMemcpyHostToDevice, st);
    // the host arrays above live on this call's stack: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = shift_estimate(&pl, X, ldx, Y, ldy, false, st);
    if (e == cudaSuccess) e = gram_f64(&pl, X, ldx, Y, ldy, st);
    if (e == cudaSuccess) e = fold_sums(&pl, st);
    if (e == cudaSuccess) e = fold_stats(&pl, flags, ddof, mean_out, std_out, st);
    if (e == cudaSuccess && (XTX || XTY)) e = epilogue(&pl, flags, XTX, XTY, st);
    return to_status(e);
}
