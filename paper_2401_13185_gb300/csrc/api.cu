// api.cu -- the C ABI declared in include/cvx.h: plan construction
// (Algorithm 1 on the device plus work decomposition), the products call
// (Algorithm 7 generalised to the 16 flag combinations) and plan queries.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "cvx_internal.cuh"

using namespace cvx;

namespace {

constexpr int64_t MIN_SEG_ROWS = 256;
// Folds averaging at most this many rows take the small-fold strategy (each
// fold's part of H recomputed from its rows in the epilogue).  Measured on
// N = 1e5, K = 500, M = 10 (FP16x3, FP32 inputs): folds of 40 and 50 rows run
// faster with the small-fold strategy (3.4 against 4.4 ms, 3.2 against
// 3.5 ms), folds of 67 rows and more fold-grouped.  cv_plan_tune measures
// both for a given problem.
constexpr int64_t SMALL_FOLD_ROWS = 64;
constexpr size_t PARTIAL_LIMIT_BYTES = size_t(24) << 30;   // scratch cap for the partial tiles
constexpr int32_t MAX_D = 1 << 15;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool split_precision(cv_precision p) {
    return p == CV_PREC_FP16X3 || p == CV_PREC_AUTO || p == CV_PREC_BF16X3 || p == CV_PREC_TF32 ||
           p == CV_PREC_TF32X3;
}

int split_kind(cv_precision p) {
    return p == CV_PREC_BF16X3   ? KIND_BF16X3
           : p == CV_PREC_TF32   ? KIND_TF32
           : p == CV_PREC_TF32X3 ? KIND_TF32X3
                                 : KIND_FP16X3;
}

struct DevFree {
    void *p = nullptr;
    ~DevFree() {
        if (p) cudaFree(p);
    }
};

cv_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CV_OK;
    if (e == cudaErrorMemoryAllocation) return CV_ERR_ALLOC;
    return CV_ERR_CUDA;
}

// Split every fold's row range into near-equal segments of at most
// rows_per_seg rows, in fold order.
void build_segments(const std::vector<int64_t> &offs, int64_t rows_per_seg,
                    std::vector<Segment> &segs, std::vector<int32_t> &fold_seg) {
    const int P = (int)offs.size() - 1;
    segs.clear();
    fold_seg.assign(P + 1, 0);
    for (int p = 0; p < P; ++p) {
        fold_seg[p] = (int32_t)segs.size();
        const int64_t nv = offs[p + 1] - offs[p];
        const int64_t k = (nv + rows_per_seg - 1) / rows_per_seg;
        for (int64_t q = 0; q < k; ++q) {
            Segment s;
            s.begin = (int32_t)(offs[p] + nv * q / k);
            s.end = (int32_t)(offs[p] + nv * (q + 1) / k);
            s.fold = p;
            s.pad = 0;
            segs.push_back(s);
        }
    }
    fold_seg[P] = (int32_t)segs.size();
}

// Segment length for the split path's tensor-core contraction, chosen by a
// model of its schedule.  Work items (segment, tile) are taken round-robin by
// G persistent CTAs in segment-major order (so the CTAs working on one
// segment's tiles run together and share its operands through L2).  An item
// of L rows costs ceil(L / 64) k-blocks of MMAs plus ITEM_KB for its
// hand-over, and every item leaves one partial tile that the fold sums read
// back, PART_KB k-block equivalents of whole-GPU memory time.  Short
// segments balance the CTAs; long ones leave fewer partial tiles.  The plan
// scans segment lengths from 256 rows up to the largest fold (at most
// max_rows) and keeps the one with the smallest (slowest CTA's k-blocks +
// items x PART_KB).  The caps:
//   FP16X3: 2^16 rows, which keeps the exact integer accumulator's scale at
//     5 bits or more;
//   BF16X3, TF32: 4096 rows (256 MMA steps), because their products
//     accumulate in FP32 inside the tensor core, where the rounding error
//     grows with the number of steps (measured: 8e-5 relative after 3125
//     steps on the 50 000-row folds of N = 1e6, P = 20).
constexpr int64_t MAX_SPLIT_SEG_ROWS = int64_t(1) << 16;
constexpr int64_t MAX_FLOAT_ACC_SEG_ROWS = 4096;

int64_t tune_rows_per_seg(const std::vector<int64_t> &offs, int ntiles, int G, int64_t max_rows) {
    constexpr double ITEM_KB = 0.3, PART_KB = 0.03;
    const int P = (int)offs.size() - 1;
    int64_t max_fold = 1;
    for (int p = 0; p < P; ++p) max_fold = std::max<int64_t>(max_fold, offs[p + 1] - offs[p]);
    max_fold = std::min(max_fold, max_rows);
    int64_t best_r = std::max<int64_t>(MIN_SEG_ROWS, max_fold);
    double best_cost = 1e300;
    std::vector<double> load(G);
    for (int64_t r = MIN_SEG_ROWS;; r = std::max<int64_t>(r + 64, r * 17 / 16)) {
        const int64_t rr = std::min(r, max_fold);
        std::fill(load.begin(), load.end(), 0.0);
        int64_t item = 0;
        for (int p = 0; p < P; ++p) {
            const int64_t nv = offs[p + 1] - offs[p];
            const int64_t k = (nv + rr - 1) / rr;
            for (int64_t q = 0; q < k; ++q) {
                const int64_t len = nv * (q + 1) / k - nv * q / k;
                const double c = (double)((len + OPS_KB - 1) / OPS_KB) + ITEM_KB;
                for (int t = 0; t < ntiles; ++t) load[(item++) % G] += c;
            }
        }
        const double cost = *std::max_element(load.begin(), load.end()) + PART_KB * (double)item;
        if (cost < best_cost) {
            best_cost = cost;
            best_r = rr;
        }
        if (rr >= max_fold) break;
    }
    return best_r;
}

// Split every owned fold's row range (folds [p_lo, p_hi)) into near-equal
// segments of at most rows_per_seg rows, in fold order; the other folds get
// no segment.
void build_segments_owned(const std::vector<int64_t> &offs, int64_t rows_per_seg, int p_lo, int p_hi,
                          std::vector<Segment> &segs, std::vector<int32_t> &fold_seg) {
    build_segments(offs, rows_per_seg, segs, fold_seg);
    const int P = (int)offs.size() - 1;
    std::vector<Segment> kept;
    std::vector<int32_t> fs(P + 1, 0);
    for (int p = 0; p < P; ++p) {
        fs[p] = (int32_t)kept.size();
        if (p >= p_lo && p < p_hi)
            for (int32_t g = fold_seg[p]; g < fold_seg[p + 1]; ++g) kept.push_back(segs[g]);
    }
    fs[P] = (int32_t)kept.size();
    segs.swap(kept);
    fold_seg.swap(fs);
}

// Flags, ddof and Definition 6's scalability check (every training partition
// holds more than ddof rows when a scale flag is set).
cv_status flags_status(const cv_plan_s *pl, int flags, int ddof) {
    const PlanView &v = pl->v;
    if (flags < 0 || flags > 15 || ddof < 0 || ddof > 1) return CV_ERR_INVALID_ARG;
    if (flags & (CV_SCALE_X | CV_SCALE_Y)) {
        for (int p = 0; p < v.P; ++p)
            if (v.N - (pl->h_offs[p + 1] - pl->h_offs[p]) - ddof < 1) return CV_ERR_NOT_SCALABLE;
    }
    return CV_OK;
}

}  // namespace

cv_status cvx::flags_arg_status(const cv_plan_s *pl, int flags, int ddof) { return flags_status(pl, flags, ddof); }

cv_status cvx::status_of(cudaError_t e) { return cuda_status(e); }

cv_status cvx::products_arg_status(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                                   int flags, int ddof) {
    if (!pl || !X) return CV_ERR_INVALID_ARG;
    const PlanView &v = pl->v;
    if (ldx < v.K) return CV_ERR_INVALID_ARG;
    if (v.M > 0 && (!Y || ldy < v.M)) return CV_ERR_INVALID_ARG;
    return flags_status(pl, flags, ddof);
}

extern "C" {

const char *cv_status_string(cv_status s) {
    switch (s) {
        case CV_OK: return "CV_OK";
        case CV_ERR_INVALID_ARG: return "CV_ERR_INVALID_ARG";
        case CV_ERR_FOLD_RANGE: return "CV_ERR_FOLD_RANGE";
        case CV_ERR_EMPTY_FOLD: return "CV_ERR_EMPTY_FOLD";
        case CV_ERR_NOT_SCALABLE: return "CV_ERR_NOT_SCALABLE";
        case CV_ERR_ALLOC: return "CV_ERR_ALLOC";
        case CV_ERR_CUDA: return "CV_ERR_CUDA";
        case CV_ERR_UNSUPPORTED: return "CV_ERR_UNSUPPORTED";
        case CV_ERR_TIMEOUT: return "CV_ERR_TIMEOUT";
        case CV_ERR_RANGE: return "CV_ERR_RANGE";
    }
    return "CV_ERR_UNKNOWN";
}

constexpr int PROF_MAX_CALLS = 4096;
constexpr int PROF_EVENTS_PER_CALL = CV_NUM_PHASES + 1;

static void free_profile_events(cv_plan_s *pl) {
    for (cudaEvent_t ev : pl->prof_events) cudaEventDestroy(ev);
    pl->prof_events.clear();
}

cv_status cv_plan_destroy(cv_plan_t plan) {
    if (!plan) return CV_OK;
    free_profile_events(plan);
    if (plan->d_block) cudaFree(plan->d_block);
    delete plan;
    return CV_OK;
}

cv_status cv_plan_profile(cv_plan_t pl, int enable) {
    if (!pl) return CV_ERR_INVALID_ARG;
    pl->prof_calls = 0;
    pl->profiling = false;
    if (!enable) return CV_OK;
    if (pl->prof_events.empty()) {
        pl->prof_events.resize((size_t)PROF_MAX_CALLS * PROF_EVENTS_PER_CALL);
        for (auto &ev : pl->prof_events) {
            if (cudaEventCreate(&ev) != cudaSuccess) {
                ev = nullptr;
                free_profile_events(pl);
                return CV_ERR_CUDA;
            }
        }
    }
    pl->profiling = true;
    return CV_OK;
}

cv_status cv_plan_phase_ms(cv_plan_t pl, double *ms, int32_t *calls) {
    if (!pl || !ms) return CV_ERR_INVALID_ARG;
    for (int k = 0; k < CV_NUM_PHASES; ++k) ms[k] = 0.0;
    const int n = pl->prof_calls;
    if (calls) *calls = n;
    if (n == 0) return CV_OK;
    if (cudaEventSynchronize(pl->prof_events[(size_t)(n - 1) * PROF_EVENTS_PER_CALL + CV_NUM_PHASES]) !=
        cudaSuccess)
        return CV_ERR_CUDA;
    for (int c = 0; c < n; ++c) {
        const cudaEvent_t *ev = &pl->prof_events[(size_t)c * PROF_EVENTS_PER_CALL];
        for (int k = 0; k < CV_NUM_PHASES; ++k) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, ev[k], ev[k + 1]) != cudaSuccess) return CV_ERR_CUDA;
            ms[k] += t;
        }
    }
    return CV_OK;
}

cv_status cv_plan(cv_plan_t *out, int64_t N, int32_t K, int32_t M, int32_t P,
                  const int32_t *fold_ids, int fold_ids_on_device, cv_dtype in_dtype,
                  cv_dtype out_dtype, cv_precision prec, void *stream) {
    return cv_plan_ex(out, N, K, M, P, fold_ids, fold_ids_on_device, in_dtype, out_dtype, prec, nullptr, stream);
}

}  // extern "C"

int64_t cvx::plan_work_units(int64_t N, int32_t K, int32_t M) {
    const int64_t nb = ((int64_t)K + M + 1 + TILE - 1) / TILE;
    return N * (nb * (nb + 1) / 2);
}

extern "C" cv_status cv_plan_ex(cv_plan_t *out, int64_t N, int32_t K, int32_t M, int32_t P,
                                const int32_t *fold_ids, int fold_ids_on_device, cv_dtype in_dtype,
                                cv_dtype out_dtype, cv_precision prec, const cv_plan_options *opts, void *stream) {
    if (!out) return CV_ERR_INVALID_ARG;
    *out = nullptr;
    const cv_plan_options o = opts ? *opts : cv_plan_options{CV_STRATEGY_AUTO, 0};
    if ((o.strategy != CV_STRATEGY_AUTO && o.strategy != CV_STRATEGY_FOLD_GROUPED &&
         o.strategy != CV_STRATEGY_SMALL_FOLDS) ||
        o.ctas < 0)
        return CV_ERR_INVALID_ARG;
    if ((o.xtx_layout != CV_XTX_FULL && o.xtx_layout != CV_XTX_PACKED_UPPER) || o.reserved != 0 ||
        o.wait_limit_ns < 0)
        return CV_ERR_INVALID_ARG;
    const bool sharded = !(o.fold_begin == 0 && o.fold_end == 0);
    if (sharded && (o.fold_begin < 0 || o.fold_begin >= o.fold_end || o.fold_end > P ||
                    o.strategy == CV_STRATEGY_SMALL_FOLDS))
        return CV_ERR_INVALID_ARG;
    // a shard keeps per-fold tiles: its folds' Grams are what it contributes
    const bool force_grouped = o.strategy == CV_STRATEGY_FOLD_GROUPED || sharded;
    if (N < 2 || N > INT32_MAX || K < 1 || M < 0 || P < 2 || (int64_t)P > N || !fold_ids)
        return CV_ERR_INVALID_ARG;
    if ((int64_t)K + M + 1 > MAX_D) return CV_ERR_INVALID_ARG;
    if ((in_dtype != CV_F32 && in_dtype != CV_F64) || (out_dtype != CV_F32 && out_dtype != CV_F64))
        return CV_ERR_INVALID_ARG;
    if (prec != CV_PREC_FP64 && !split_precision(prec)) return CV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cv_plan_s *pl = new (std::nothrow) cv_plan_s();
    if (!pl) return CV_ERR_ALLOC;
    pl->in_dtype = in_dtype;
    pl->out_dtype = out_dtype;
    pl->prec = prec;
    pl->opts = o;
    pl->d_block = nullptr;
    pl->ypack = nullptr;
    pl->ypack_width = 0;
    pl->profiling = false;
    pl->prof_calls = 0;
    pl->launches = 0;
    pl->has_sums = false;
    pl->sharded = sharded;
    pl->has_partial = false;
    pl->gathered = false;
    cudaError_t e = cudaGetDevice(&pl->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device);
    if (e != cudaSuccess) {
        delete pl;
        return CV_ERR_CUDA;
    }

    PlanView &v = pl->v;
    memset(&v, 0, sizeof(v));
    v.N = N;
    v.K = K;
    v.M = M;
    v.P = P;
    v.D = K + M + 1;
    v.nb = (v.D + TILE - 1) / TILE;
    v.ntiles = v.nb * (v.nb + 1) / 2;
    v.nlast = std::min(TILE, (v.D - TILE * (v.nb - 1) + 15) / 16 * 16);
    v.p_lo = sharded ? o.fold_begin : 0;
    v.p_hi = sharded ? o.fold_end : P;
    v.packed = o.xtx_layout == CV_XTX_PACKED_UPPER ? 1 : 0;
    v.wait_ns = o.wait_limit_ns > 0 ? (uint64_t)o.wait_limit_ns : 1000000000ull;

    // ---- Algorithm 1, step 1: validate ids and count rows per fold --------
    DevFree d_tmp_folds, d_counts;
    const int32_t *d_folds = fold_ids;
    if (!fold_ids_on_device) {
        if ((e = cudaMalloc(&d_tmp_folds.p, sizeof(int32_t) * N)) != cudaSuccess) {
            delete pl;
            return cuda_status(e);
        }
        e = cudaMemcpyAsync(d_tmp_folds.p, fold_ids, sizeof(int32_t) * N, cudaMemcpyHostToDevice, st);
        d_folds = (const int32_t *)d_tmp_folds.p;
    }
    const size_t count_bytes = sizeof(unsigned long long) * P + sizeof(int);
    if (e == cudaSuccess) e = cudaMalloc(&d_counts.p, count_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counts.p, 0, count_bytes, st);
    unsigned long long *d_cnt = (unsigned long long *)d_counts.p;
    int *d_bad = (int *)(d_cnt + P);
    if (e == cudaSuccess) e = fold_count(d_folds, N, P, d_cnt, d_bad, st);
    std::vector<unsigned long long> counts(P);
    int bad = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(counts.data(), d_cnt, sizeof(unsigned long long) * P, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        delete pl;
        return cuda_status(e);
    }
    if (bad) {
        delete pl;
        return CV_ERR_FOLD_RANGE;
    }
    pl->h_offs.assign(P + 1, 0);
    for (int p = 0; p < P; ++p) {
        if (counts[p] == 0) {
            delete pl;
            return CV_ERR_EMPTY_FOLD;
        }
        pl->h_offs[p + 1] = pl->h_offs[p] + (int64_t)counts[p];
    }

    // ---- work decomposition: segments x upper-triangle tiles -------------
    const bool split = split_precision(prec);
    const bool small = o.strategy == CV_STRATEGY_SMALL_FOLDS || (!force_grouped && N <= SMALL_FOLD_ROWS * (int64_t)P);
    const int ctas = o.ctas > 0 ? o.ctas : pl->num_sms;   // what the segments are tuned for
    const int64_t target_items = (int64_t)4 * ctas;
    int64_t rows_per_seg = std::max<int64_t>(MIN_SEG_ROWS, (N * v.ntiles + target_items - 1) / target_items);
    if (split && !small)
        rows_per_seg = tune_rows_per_seg(pl->h_offs, v.ntiles, ctas,
                                         split_kind(prec) == KIND_FP16X3 ? MAX_SPLIT_SEG_ROWS : MAX_FLOAT_ACC_SEG_ROWS);
    std::vector<int32_t> fold_seg;
    if (small) {   // segments over all rows, one pseudo-fold: only H over all rows is reduced
        const std::vector<int64_t> all = {0, N};
        build_segments(all, rows_per_seg, pl->h_segs, fold_seg);
    } else {
        build_segments(pl->h_offs, rows_per_seg, pl->h_segs, fold_seg);
    }
    // The operand scale below depends on the longest segment of ALL folds, so
    // that every shard of a fold-sharded computation scales alike; only then
    // are a shard's segments cut down to its own folds.
    int64_t longest_seg = 1;
    for (const Segment &sg : pl->h_segs) longest_seg = std::max<int64_t>(longest_seg, sg.end - sg.begin);
    if (sharded) build_segments_owned(pl->h_offs, rows_per_seg, v.p_lo, v.p_hi, pl->h_segs, fold_seg);
    v.nsegs = (int32_t)pl->h_segs.size();
    // Split precision: the integer part of every scaled value is summed exactly
    // in FP32 while a segment's sum of hi * hi stays below 2^24.  With the
    // sampled maximum at 2^B and a typical value near 2^B / 3.5 that needs
    // L * 2^(2B) / 12.25 < 2^23 for the longest segment of L rows.
    {
        const int64_t L = (int64_t)align_up((size_t)longest_seg, 64);
        int b = (int)std::floor((23.0 + std::log2(12.25) - std::log2((double)L)) / 2.0);
        v.int_bits = std::max(4, std::min(10, b));   // FP16 holds integers exactly up to 2^11
    }
    // Narrow last-block tiles cost a quarter of a full tile or less, so the
    // CTAs that take them run ahead of the others on the same segment.  With
    // segments whose operands do not fit in L2 together (the FP16X3 path's
    // long segments), that breaks the shared L2 reads of the segment's tiles:
    // measured 2.79 ms against 2.65 ms for full-width tiles on N = 1e6,
    // K = 1024, M = 16.  Short segments (at most 4096 rows) keep them narrow.
    if (split && longest_seg > MAX_FLOAT_ACC_SEG_ROWS) v.nlast = TILE;
    std::vector<TileCoord> tiles;
    for (int bi = 0; bi < v.nb; ++bi)
        for (int bj = bi; bj < v.nb; ++bj) tiles.push_back(TileCoord{bi, bj});

    const size_t partial_bytes = (size_t)v.nsegs * v.ntiles * TILE_ELEMS * sizeof(double);
    const size_t tile_bytes = (size_t)ops_tile_bytes(split_kind(prec));
    const size_t ops_bytes_est = split ? ((size_t)N / OPS_KB + 2 * v.nsegs) * v.nb * tile_bytes : 0;
    const size_t g_elem = split ? sizeof(long long) + sizeof(float) : sizeof(double);
    // fold sums: FP64 path only (the split path forms them from the partials)
    const size_t gfold_bytes = small || split ? 0 : (size_t)P * v.ntiles * TILE_ELEMS * g_elem;
    if (partial_bytes + ops_bytes_est + gfold_bytes + (size_t)v.ntiles * TILE_ELEMS * g_elem >
        PARTIAL_LIMIT_BYTES) {
        delete pl;
        return CV_ERR_UNSUPPORTED;
    }

    // ---- workspace layout -------------------------------------------------
    const int KM = K + M;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_perm = carve(sizeof(int32_t) * N);
    const size_t o_offs = carve(sizeof(int64_t) * (P + 1));
    const size_t o_segs = carve(sizeof(Segment) * v.nsegs);
    const size_t o_fseg = carve(sizeof(int32_t) * fold_seg.size());
    const size_t o_tiles = carve(sizeof(TileCoord) * v.ntiles);
    const size_t o_part = carve(partial_bytes);
    const size_t o_gfold = carve(gfold_bytes);
    const size_t o_gtot = carve((size_t)v.ntiles * TILE_ELEMS * g_elem);
    const size_t o_shift = carve(sizeof(double) * v.D);
    const size_t o_isc = carve(sizeof(double) * v.D);
    const size_t o_shf = carve(sizeof(float) * v.D);
    const size_t o_scf = carve(sizeof(float) * v.D);
    const size_t o_stats = carve(sizeof(double) * 4 * (size_t)P * KM);
    const size_t o_facf = split ? carve(sizeof(float4) * (size_t)P * KM) : 0;
    const size_t o_fact = split ? carve(sizeof(int32_t) * (size_t)P * KM) : 0;
    const size_t o_fsq = small ? carve((split ? sizeof(float2) : sizeof(double2)) * (size_t)P * KM) : 0;
    v.nsample = (int32_t)std::min<int64_t>(N, SHIFT_SAMPLE);
    const size_t o_err = carve(sizeof(int) * 4);
    // split precision: k-block table and the converted operand tiles
    std::vector<KBlock> kblocks;
    std::vector<int32_t> seg_kb;
    size_t o_kb = 0, o_segkb = 0, o_ops = 0;
    if (split) {
        seg_kb.reserve(v.nsegs + 1);
        for (const Segment &sg : pl->h_segs) {
            seg_kb.push_back((int32_t)kblocks.size());
            for (int32_t r = sg.begin; r < sg.end; r += OPS_KB)
                kblocks.push_back(KBlock{r, std::min<int32_t>(OPS_KB, sg.end - r)});
        }
        seg_kb.push_back((int32_t)kblocks.size());
        v.nkb = (int32_t)kblocks.size();
        o_kb = carve(sizeof(KBlock) * kblocks.size());
        o_segkb = carve(sizeof(int32_t) * seg_kb.size());
        o_ops = carve((size_t)v.nkb * v.nb * tile_bytes);
    }
    size_t o_ypack = 0;
    pl->ypack = nullptr;
    pl->ypack_width = 0;
    if (split && in_dtype == CV_F32) {
        pl->ypack_width = (int)align_up((size_t)M + 1, 4);
        o_ypack = carve(sizeof(float) * (size_t)N * pl->ypack_width);
    }
    pl->ws_bytes = off;
    if ((e = cudaMalloc(&pl->d_block, off)) != cudaSuccess) {
        delete pl;
        return cuda_status(e);
    }
    char *base = (char *)pl->d_block;
    v.perm = (int32_t *)(base + o_perm);
    v.offs = (int64_t *)(base + o_offs);
    v.segs = (Segment *)(base + o_segs);
    v.fold_seg = (int32_t *)(base + o_fseg);
    v.tiles = (TileCoord *)(base + o_tiles);
    v.partials = (double *)(base + o_part);
    v.split = split ? 1 : 0;
    v.kind = split_kind(prec);
    v.small = small ? 1 : 0;
    v.gfold = small || split ? nullptr : (void *)(base + o_gfold);
    v.fold_sq = small ? (void *)(base + o_fsq) : nullptr;
    v.gtot = (void *)(base + o_gtot);
    v.sp.shift = (double *)(base + o_shift);
    v.sp.inv_scale = (double *)(base + o_isc);
    v.sp.shift_f = (float *)(base + o_shf);
    v.sp.scale_f = (float *)(base + o_scf);
    v.stats = (double *)(base + o_stats);
    v.fac_f = split ? (float4 *)(base + o_facf) : nullptr;
    v.fac_t = split ? (int32_t *)(base + o_fact) : nullptr;
    v.err = (int *)(base + o_err);
    if (split) {
        v.kblocks = (KBlock *)(base + o_kb);
        v.seg_kb = (int32_t *)(base + o_segkb);
        v.ops = (void *)(base + o_ops);
    }
    if (pl->ypack_width) pl->ypack = (float *)(base + o_ypack);

    // ---- Algorithm 1, steps 2-5: stable scatter of rows by fold ---------
    DevFree d_sort_tmp;
    const size_t tmp_bytes = fold_sort_tmp_bytes(N);
    e = cudaMalloc(&d_sort_tmp.p, tmp_bytes);
    if (e == cudaSuccess) e = fold_sort(d_folds, N, P, v.perm, d_sort_tmp.p, tmp_bytes, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(v.offs, pl->h_offs.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(v.segs, pl->h_segs.data(), sizeof(Segment) * v.nsegs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(v.fold_seg, fold_seg.data(), sizeof(int32_t) * fold_seg.size(), cudaMemcpyHostToDevice,
                            st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(v.tiles, tiles.data(), sizeof(TileCoord) * v.ntiles, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && split) {
        e = cudaMemcpyAsync(v.kblocks, kblocks.data(), sizeof(KBlock) * kblocks.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(v.seg_kb, seg_kb.data(), sizeof(int32_t) * seg_kb.size(), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(v.err, 0, sizeof(int) * 4, st);
    // how often the fold-sorted order breaks a run of consecutive rows (the
    // count buffer's first word is free again)
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = perm_breaks(v.perm, N, d_cnt, st);
    // Split path: the columns of the last block past nlast are neither
    // converted nor contracted; zeroed once here, the operand tiles and the
    // partial tiles hold zeros there for the plan's lifetime.
    if (e == cudaSuccess && split) e = cudaMemsetAsync(v.ops, 0, (size_t)v.nkb * v.nb * tile_bytes, st);
    if (e == cudaSuccess && split) e = cudaMemsetAsync(v.partials, 0, partial_bytes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    unsigned long long breaks = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&breaks, d_cnt, sizeof(breaks), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cv_plan_destroy(pl);
        return cuda_status(e);
    }
    // more than one break per 8 k-blocks of 64 rows on average
    pl->gathered = breaks * 512 > (unsigned long long)N;
    *out = pl;
    return CV_OK;
}

extern "C" {

cv_status cv_products(cv_plan_t pl, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                      int flags, int ddof, void *XTX, void *XTY, double *mean_out, double *std_out,
                      void *stream) {
    const cv_status chk = cvx::products_arg_status(pl, X, ldx, Y, ldy, flags, ddof);
    if (chk != CV_OK) return chk;
    if (pl->sharded) return CV_ERR_INVALID_ARG;   // cv_products_partial + cv_finalize_total
    const PlanView &v = pl->v;
    cudaStream_t st = (cudaStream_t)stream;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return CV_ERR_CUDA;
    if (cur != pl->device && cudaSetDevice(pl->device) != cudaSuccess) return CV_ERR_CUDA;
    const bool split = split_precision(pl->prec);
    cudaEvent_t *ev = nullptr;
    if (pl->profiling && pl->prof_calls < PROF_MAX_CALLS)
        ev = &pl->prof_events[(size_t)(pl->prof_calls++) * PROF_EVENTS_PER_CALL];
    auto mark = [&](int k) {
        if (ev) cudaEventRecord(ev[k], st);
    };
    mark(0);
    cudaError_t e = shift_estimate(pl, X, ldx, Y, ldy, split, st);
    mark(1);
    if (e == cudaSuccess && split) e = convert_split(pl, X, ldx, Y, ldy, st);
    mark(2);
    if (e == cudaSuccess) e = split ? gram_tc(pl, st) : gram_f64(pl, X, ldx, Y, ldy, st);
    mark(3);
    const bool tail = fused_tail(pl);
    if (e == cudaSuccess && !tail) e = fold_sums(pl, st);
    if (e == cudaSuccess && v.small) e = small_fold_colsums(pl, X, ldx, Y, ldy, st);
    mark(4);
    if (e == cudaSuccess) e = tail ? split_stats(pl, flags, ddof, mean_out, std_out, st)
                                   : fold_stats(pl, flags, ddof, mean_out, std_out, st);
    mark(5);
    if (e == cudaSuccess && (XTX || XTY))
        e = v.small ? small_fold_epilogue(pl, flags, X, ldx, Y, ldy, XTX, XTY, st)
                    : tail ? fold_epilogue_split(pl, flags, XTX, XTY, st) : epilogue(pl, flags, XTX, XTY, st);
    mark(6);
    if (cur != pl->device) cudaSetDevice(cur);
    if (e == cudaSuccess) pl->has_sums = true;
    if (e == cudaErrorNotSupported) return CV_ERR_UNSUPPORTED;
    return cuda_status(e);
}

cv_status cv_finalize(cv_plan_t pl, const void *X, int64_t ldx, const void *Y, int64_t ldy, int flags, int ddof,
                      void *XTX, void *XTY, double *mean_out, double *std_out, void *stream) {
    if (!pl || !pl->has_sums) return CV_ERR_INVALID_ARG;
    const PlanView &v = pl->v;
    // the small-fold strategy recomputes each fold's part from the rows
    const cv_status chk = v.small ? cvx::products_arg_status(pl, X, ldx, Y, ldy, flags, ddof)
                                  : flags_status(pl, flags, ddof);
    if (chk != CV_OK) return chk;
    cudaStream_t st = (cudaStream_t)stream;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return CV_ERR_CUDA;
    if (cur != pl->device && cudaSetDevice(pl->device) != cudaSuccess) return CV_ERR_CUDA;
    const bool tail = fused_tail(pl);
    cudaError_t e = tail ? split_stats(pl, flags, ddof, mean_out, std_out, st)
                         : fold_stats(pl, flags, ddof, mean_out, std_out, st);
    if (e == cudaSuccess && (XTX || XTY))
        e = v.small ? small_fold_epilogue(pl, flags, X, ldx, Y, ldy, XTX, XTY, st)
                    : tail ? fold_epilogue_split(pl, flags, XTX, XTY, st) : epilogue(pl, flags, XTX, XTY, st);
    if (cur != pl->device) cudaSetDevice(cur);
    return cuda_status(e);
}

cv_status cv_plan_status(cv_plan_t pl, void *stream) {
    if (!pl) return CV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int err = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&err, pl->v.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(pl->v.err, 0, sizeof(int));
    if (e != cudaSuccess) return CV_ERR_CUDA;
    if (err & DEV_ERR_TIMEOUT) return CV_ERR_TIMEOUT;
    if (err & DEV_ERR_RANGE) return CV_ERR_RANGE;
    return CV_OK;
}

cv_status cv_plan_fold_offsets(cv_plan_t pl, int64_t *offsets) {
    if (!pl || !offsets) return CV_ERR_INVALID_ARG;
    memcpy(offsets, pl->h_offs.data(), sizeof(int64_t) * pl->h_offs.size());
    return CV_OK;
}

cv_status cv_plan_permutation(cv_plan_t pl, int32_t *perm) {
    if (!pl || !perm) return CV_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpy(perm, pl->v.perm, sizeof(int32_t) * pl->v.N, cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

cv_status cv_plan_launches(cv_plan_t pl, int64_t *count) {
    if (!pl || !count) return CV_ERR_INVALID_ARG;
    *count = pl->launches;
    return CV_OK;
}

cv_status cv_plan_workspace_bytes(cv_plan_t pl, int64_t *bytes) {
    if (!pl || !bytes) return CV_ERR_INVALID_ARG;
    *bytes = (int64_t)pl->ws_bytes;
    return CV_OK;
}

}  // extern "C"
