// batch.cu -- batches of independent cross-validation problems.
//
// Each problem keeps its own plan (Algorithm 1 and workspace).  Two ways to
// run a batch's products:
//
//   Batched launches (tensor-core precisions, FP32 inputs, at most 32 folds
//   per problem): every stage of the path runs as ONE launch over all
//   problems' work units -- shift estimate (one 8-CTA cluster per problem and
//   column group), operand conversion (one block per problem and run of
//   k-blocks, whole rows), the persistent contraction (the (problem, item) pairs of
//   all plans assigned to the CTAs longest first), the statistics from the
//   segment partials, and the fused fold-sum + epilogue (one launch per class
//   of fold counts, P <= 8, <= 16, <= 32, so that each sizes its shared memory
//   for its own folds).  Five to seven launches for the whole batch; the
//   plans are made with the fold-grouped strategy so that
//   every problem takes the same kernels.  The work tables are built once, in
//   cv_batch_plan; each call passes the problems' pointers, flags and ddof as
//   a kernel parameter (batches of at most 256 problems: nothing is copied
//   and the call can be captured into a CUDA graph) or copies them to the
//   device (larger batches).
//
//   A CUDA graph (otherwise): a fork event on an internal origin stream, every
//   problem's cv_products on one of up to 32 internal worker streams (in
//   decreasing order of work, round-robin), and a join back to the origin.  The
//   graph is kept and relaunched while the problem descriptors stay the same;
//   a changed descriptor triggers a re-capture, applied as an in-place update
//   of the executable graph when its topology allows.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "cvx_internal.cuh"

struct cv_batch_s {
    // batched launches
    bool fused = false;
    cvx::BatchTables tables = {};
    void *d_tables = nullptr;                 // device copy of the views and work units
    cvx::ProblemArgs *d_args = nullptr;       // this call's per-problem arguments (device)
    cvx::ProblemArgs *h_args = nullptr;       // their pinned host staging
    cudaEvent_t args_copied = nullptr;        // the staging may be rewritten after this
    bool args_valid = false;                  // d_args holds the arguments of the last call
    cvx::BatchArgs *kargs = nullptr;          // batches of at most BATCH_ARGS_MAX problems: the
                                              // arguments as a kernel parameter (host copy)
    // epilogue launches: one per fold-count class, each with shared memory for
    // its own largest P (units of the class are contiguous in the table)
    struct EpiClass {
        int32_t begin, count, max_P;
    };
    std::vector<EpiClass> epi_classes;
    int64_t launches = 0;                     // kernels enqueued by cv_batch_products
    int64_t graph_launches = 0;               // kernels in the captured graph
    std::vector<cv_plan_t> plans;
    std::vector<cv_plan_options> opts;  // each problem's plan options
    std::vector<cv_problem> shapes;     // descriptors as planned
    std::vector<cudaStream_t> workers;
    std::vector<cudaEvent_t> joins;     // one per worker
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cv_problem> captured;   // descriptors the graph was captured with
    std::vector<int> order;             // problems by decreasing N K (K + M)
};

namespace {

constexpr int BATCH_STREAMS = 32;

void release(cv_batch_s *b) {
    delete b->kargs;
    if (b->args_copied) cudaEventDestroy(b->args_copied);
    if (b->h_args) cudaFreeHost(b->h_args);
    if (b->d_tables) cudaFree(b->d_tables);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
    for (cudaStream_t s : b->workers) cudaStreamDestroy(s);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->origin) cudaStreamDestroy(b->origin);
    for (cv_plan_t p : b->plans) cv_plan_destroy(p);
    delete b;
}

bool same_problem(const cv_problem &a, const cv_problem &b) {
    return a.N == b.N && a.K == b.K && a.M == b.M && a.P == b.P && a.fold_ids == b.fold_ids && a.X == b.X &&
           a.ldx == b.ldx && a.Y == b.Y && a.ldy == b.ldy && a.flags == b.flags && a.ddof == b.ddof &&
           a.XTX == b.XTX && a.XTY == b.XTY && a.mean_out == b.mean_out && a.std_out == b.std_out;
}

cv_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return CV_OK;
    return e == cudaErrorMemoryAllocation ? CV_ERR_ALLOC : CV_ERR_CUDA;
}

// Capture every problem's cv_products into a graph rooted on the origin stream.
cv_status capture(cv_batch_s *b, const cv_problem *probs, cudaGraph_t *graph) {
    const int count = (int)b->plans.size();
    const int ns = (int)b->workers.size();
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return to_status(e);
    cv_status st = CV_OK;
    e = cudaEventRecord(b->fork, b->origin);
    for (int w = 0; w < ns && e == cudaSuccess; ++w) e = cudaStreamWaitEvent(b->workers[w], b->fork, 0);
    // longest first: each branch takes the next problem in decreasing order of
    // algorithmic work N K (K + M), so the large problems do not end up alone
    // at the tail of the graph
    for (int r = 0; r < count && e == cudaSuccess && st == CV_OK; ++r) {
        const int i = b->order[r];
        const cv_problem &q = probs[i];
        st = cv_products(b->plans[i], q.X, q.ldx, q.Y, q.ldy, q.flags, q.ddof, q.XTX, q.XTY, q.mean_out, q.std_out,
                         b->workers[r % ns]);
    }
    for (int w = 0; w < ns && e == cudaSuccess && st == CV_OK; ++w) {
        e = cudaEventRecord(b->joins[w], b->workers[w]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->joins[w], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(b->origin, &g);
    if (st == CV_OK && e == cudaSuccess && e_end == cudaSuccess) {
        *graph = g;
        return CV_OK;
    }
    if (g) cudaGraphDestroy(g);
    if (st != CV_OK) return st;
    return to_status(e != cudaSuccess ? e : e_end);
}

// Fold-count class of a problem for the epilogue launches: P <= 8, <= 16, <= 32.
int epi_class(int P) { return P <= 8 ? 0 : (P <= 16 ? 1 : 2); }

// The work tables of the batched launches (see the top of this file).
cv_status build_tables(cv_batch_s *b, cv_dtype out_dtype, cudaStream_t st) {
    const int count = (int)b->plans.size();
    int num_sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CV_ERR_CUDA;
    std::vector<cvx::PlanView> views(count);
    std::vector<int2> shift_units, gram_items;
    std::vector<int4> conv_units, stats_units, epi_units;
    std::vector<std::pair<double, int2>> items;   // (cost in k-blocks, (problem, item))
    int max_P = 1;
    for (int i = 0; i < count; ++i) {
        const cvx::PlanView &v = b->plans[i]->v;
        views[i] = v;
        max_P = std::max(max_P, v.P);
        for (int g = 0; g < (v.D + 31) / 32; ++g) shift_units.push_back(make_int2(i, g));
        // conversion: runs of k-blocks of about 8192 (16-row group, column) pairs each
        const int run = cvx::direct_run(v.D);
        for (int g0 = 0; g0 < v.nkb; g0 += run) conv_units.push_back(make_int4(i, g0, std::min(v.nkb, g0 + run), 0));
        const std::vector<cvx::Segment> &segs = b->plans[i]->h_segs;
        for (int sgi = 0; sgi < v.nsegs; ++sgi) {
            const double kb = (double)((segs[sgi].end - segs[sgi].begin + cvx::OPS_KB - 1) / cvx::OPS_KB) + 0.3;
            for (int t = 0; t < v.ntiles; ++t) items.push_back({kb, make_int2(i, sgi * v.ntiles + t)});
        }
        for (int c0 = 0; c0 < v.K + v.M; c0 += 32)
            for (int p = 0; p < v.P; ++p) stats_units.push_back(make_int4(i, c0, p, 0));
        int t = 0;   // tiles in the plan's enumeration: row-major upper block triangle
        for (int bi = 0; bi < v.nb; ++bi)
            for (int bj = bi; bj < v.nb; ++bj, ++t)
                for (int sub = 0; sub < 64; ++sub) {
                    const int i0 = bi * cvx::TILE + 16 * (sub / 8), j0 = bj * cvx::TILE + 16 * (sub % 8);
                    if (i0 < v.K && j0 < v.K + v.M && j0 + 15 >= i0)
                        epi_units.push_back(make_int4(i, t, sub, epi_class(v.P)));
                }
    }
    // epilogue units grouped by fold-count class, largest class first
    std::stable_sort(epi_units.begin(), epi_units.end(), [](const int4 &x, const int4 &y) { return x.w > y.w; });
    for (size_t k = 0; k < epi_units.size(); ++k) {
        const int P = b->plans[epi_units[k].x]->v.P;
        if (b->epi_classes.empty() || epi_units[k].w != epi_units[k - 1].w)
            b->epi_classes.push_back({(int32_t)k, 0, 0});
        ++b->epi_classes.back().count;
        b->epi_classes.back().max_P = std::max(b->epi_classes.back().max_P, P);
    }
    // longest first onto the least-loaded CTA
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, int2> &x, const std::pair<double, int2> &y) { return x.first > y.first; });
    const int G = std::max(1, std::min<int>(num_sms, (int)items.size()));
    std::vector<double> load(G, 0.0);
    std::vector<std::vector<int2>> per_cta(G);
    for (const auto &it : items) {
        const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[c] += it.first;
        per_cta[c].push_back(it.second);
    }
    std::vector<int32_t> gram_cta(G + 1, 0);
    for (int c = 0; c < G; ++c) {
        gram_cta[c + 1] = gram_cta[c] + (int32_t)per_cta[c].size();
        gram_items.insert(gram_items.end(), per_cta[c].begin(), per_cta[c].end());
    }
    // one device block: views, args, units
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_views = carve(sizeof(cvx::PlanView) * count);
    const size_t o_args = carve(sizeof(cvx::ProblemArgs) * count);
    const size_t o_shift = carve(sizeof(int2) * shift_units.size());
    const size_t o_conv = carve(sizeof(int4) * conv_units.size());
    const size_t o_items = carve(sizeof(int2) * gram_items.size());
    const size_t o_cta = carve(sizeof(int32_t) * gram_cta.size());
    const size_t o_stats = carve(sizeof(int4) * stats_units.size());
    const size_t o_epi = carve(sizeof(int4) * epi_units.size());
    b->kargs = new (std::nothrow) cvx::BatchArgs();
    if (!b->kargs) return CV_ERR_ALLOC;
    cudaError_t e = cudaMalloc(&b->d_tables, off);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_args, sizeof(cvx::ProblemArgs) * count);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->args_copied, cudaEventDisableTiming);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CV_ERR_ALLOC : CV_ERR_CUDA;
    char *base = (char *)b->d_tables;
    auto up = [&](size_t o, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, st);
    };
    up(o_views, views.data(), sizeof(cvx::PlanView) * count);
    up(o_shift, shift_units.data(), sizeof(int2) * shift_units.size());
    up(o_conv, conv_units.data(), sizeof(int4) * conv_units.size());
    up(o_items, gram_items.data(), sizeof(int2) * gram_items.size());
    up(o_cta, gram_cta.data(), sizeof(int32_t) * gram_cta.size());
    up(o_stats, stats_units.data(), sizeof(int4) * stats_units.size());
    up(o_epi, epi_units.data(), sizeof(int4) * epi_units.size());
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host vectors go out of scope
    if (e != cudaSuccess) return CV_ERR_CUDA;
    cvx::BatchTables &bt = b->tables;
    bt.views = (const cvx::PlanView *)(base + o_views);
    b->d_args = (cvx::ProblemArgs *)(base + o_args);
    bt.args = b->d_args;
    bt.shift_units = (const int2 *)(base + o_shift);
    bt.n_shift = (int32_t)shift_units.size();
    bt.conv_units = (const int4 *)(base + o_conv);
    bt.n_conv = (int32_t)conv_units.size();
    bt.gram_items = (const int2 *)(base + o_items);
    bt.gram_cta = (const int32_t *)(base + o_cta);
    bt.gram_ctas = G;
    bt.stats_units = (const int4 *)(base + o_stats);
    bt.n_stats = (int32_t)stats_units.size();
    bt.epi_units = (const int4 *)(base + o_epi);
    bt.n_epi = (int32_t)epi_units.size();
    bt.max_P = max_P;
    bt.kind = views[0].kind;
    bt.out_f64 = out_dtype == CV_F64 ? 1 : 0;
    b->fused = true;
    return CV_OK;
}

// One call's products through the batched launches.
cv_status run_fused(cv_batch_s *b, const cv_problem *probs, cudaStream_t st) {
    const int count = (int)b->plans.size();
    std::vector<cvx::ProblemArgs> args(count);
    for (int i = 0; i < count; ++i) {
        const cv_problem &q = probs[i];
        cvx::ProblemArgs &a = args[i];
        a.X = q.X;
        a.Y = q.Y;
        a.ldx = q.ldx;
        a.ldy = q.ldy;
        a.XTX = q.XTX;
        a.XTY = q.XTY;
        a.mean_out = q.mean_out;
        a.std_out = q.std_out;
        a.flags = q.flags;
        a.ddof = q.ddof;
        a.x_vec = ((uintptr_t)q.X % 16 == 0) && (q.ldx % 4 == 0);
        a.pad = 0;
    }
    cudaError_t e = cudaSuccess;
    cvx::BatchTables tables = b->tables;
    if (count <= cvx::BATCH_ARGS_MAX) {
        // the arguments travel as a kernel parameter: no copy, no host wait,
        // so the call can be captured into a CUDA graph
        std::memcpy(b->kargs->a, args.data(), sizeof(cvx::ProblemArgs) * count);
        tables.args = nullptr;
    } else if (!b->args_valid || std::memcmp(args.data(), b->h_args, sizeof(cvx::ProblemArgs) * count) != 0) {
        // a repeated call with the same arguments reuses the device copy;
        // otherwise the staging is rewritten once the previous call's copy
        // has been made
        b->args_valid = false;
        e = cudaEventSynchronize(b->args_copied);
        if (e == cudaSuccess) {
            std::memcpy(b->h_args, args.data(), sizeof(cvx::ProblemArgs) * count);
            e = cudaMemcpyAsync(b->d_args, b->h_args, sizeof(cvx::ProblemArgs) * count, cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess) e = cudaEventRecord(b->args_copied, st);
        if (e != cudaSuccess) return to_status(e);
        b->args_valid = true;
    }
    const cvx::BatchArgs &ka = *b->kargs;   // unused by the kernels when tables.args is set
    b->launches += 4 + (int64_t)b->epi_classes.size();
    if (e == cudaSuccess) e = cvx::shift_estimate_batched(tables, ka, st);
    if (e == cudaSuccess) e = cvx::convert_batched(tables, ka, st);
    if (e == cudaSuccess) e = cvx::gram_tc_batched(tables, st);
    if (e == cudaSuccess) e = cvx::split_stats_batched(tables, ka, st);
    for (const auto &ec : b->epi_classes) {
        if (e != cudaSuccess) break;
        cvx::BatchTables t = tables;
        t.epi_units += ec.begin;
        t.n_epi = ec.count;
        t.max_P = ec.max_P;
        e = cvx::fold_epilogue_split_batched(t, ka, st);
    }
    return to_status(e);
}

}  // namespace

extern "C" {

cv_status cv_batch_plan(cv_batch_t *out, const cv_problem *probs, int32_t count, int fold_ids_on_device,
                        cv_dtype in_dtype, cv_dtype out_dtype, cv_precision prec, void *stream) {
    if (!out) return CV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!probs || count < 1) return CV_ERR_INVALID_ARG;
    cv_batch_s *b = new (std::nothrow) cv_batch_s();
    if (!b) return CV_ERR_ALLOC;
    // batched launches: a tensor-core precision, FP32 inputs, at most
    // BATCH_FOLD_MAX folds in every problem
    bool fused = prec != CV_PREC_FP64 && in_dtype == CV_F32;
    for (int i = 0; i < count && fused; ++i) fused = probs[i].P <= cvx::BATCH_FOLD_MAX;
    // each problem's segments are tuned for its share of the SMs, in
    // proportion to its contraction work
    int num_sms = 1, dev = 0;
    if (fused && (cudaGetDevice(&dev) != cudaSuccess ||
                  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)) {
        release(b);
        return CV_ERR_CUDA;
    }
    double total_work = 0.0;
    for (int i = 0; i < count; ++i) total_work += (double)cvx::plan_work_units(probs[i].N, probs[i].K, probs[i].M);
    b->opts.resize(count, cv_plan_options{CV_STRATEGY_AUTO, 0});
    for (int i = 0; i < count; ++i) {
        const cv_problem &q = probs[i];
        if (fused) {
            const double share = num_sms * (double)cvx::plan_work_units(q.N, q.K, q.M) / std::max(1.0, total_work);
            b->opts[i] = cv_plan_options{CV_STRATEGY_FOLD_GROUPED, std::max(1, (int)share)};
        }
        cv_plan_t p = nullptr;
        const cv_status st = cv_plan_ex(&p, q.N, q.K, q.M, q.P, q.fold_ids, fold_ids_on_device, in_dtype, out_dtype,
                                        prec, &b->opts[i], stream);
        if (st != CV_OK) {
            release(b);
            return st;
        }
        b->plans.push_back(p);
        b->shapes.push_back(q);
    }
    b->order.resize(count);
    for (int i = 0; i < count; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        const double wx = (double)probs[x].N * probs[x].K * (probs[x].K + probs[x].M);
        const double wy = (double)probs[y].N * probs[y].K * (probs[y].K + probs[y].M);
        return wx > wy;
    });
    const int ns = std::min<int>(count, BATCH_STREAMS);
    cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int w = 0; w < ns && e == cudaSuccess; ++w) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->workers.push_back(s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->joins.push_back(ev);
    }
    if (e != cudaSuccess) {
        release(b);
        return to_status(e);
    }
    if (fused) {
        const cv_status st = build_tables(b, out_dtype, (cudaStream_t)stream);
        if (st != CV_OK) {
            release(b);
            return st;
        }
    }
    *out = b;
    return CV_OK;
}

cv_status cv_batch_products(cv_batch_t b, const cv_problem *probs, void *stream) {
    if (!b || !probs) return CV_ERR_INVALID_ARG;
    const int count = (int)b->plans.size();
    for (int i = 0; i < count; ++i) {
        const cv_problem &q = probs[i], &s = b->shapes[i];
        if (q.N != s.N || q.K != s.K || q.M != s.M || q.P != s.P) return CV_ERR_INVALID_ARG;
        const cv_status chk = cvx::products_arg_status(b->plans[i], q.X, q.ldx, q.Y, q.ldy, q.flags, q.ddof);
        if (chk != CV_OK) return chk;
    }
    if (b->fused) return run_fused(b, probs, (cudaStream_t)stream);
    bool same = b->exec && b->captured.size() == (size_t)count;
    for (int i = 0; same && i < count; ++i) same = same_problem(b->captured[i], probs[i]);
    if (!same) {
        int64_t before = 0, after = 0, n = 0;
        for (cv_plan_t p : b->plans) before += (cv_plan_launches(p, &n), n);
        cudaGraph_t g = nullptr;
        const cv_status st = capture(b, probs, &g);
        for (cv_plan_t p : b->plans) after += (cv_plan_launches(p, &n), n);
        b->graph_launches = after - before;
        if (st != CV_OK) return st;
        if (b->exec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(b->exec, g, &info) != cudaSuccess) {
                cudaGetLastError();   // the failed update is not sticky
                cudaGraphExecDestroy(b->exec);
                b->exec = nullptr;
            }
        }
        cudaError_t e = cudaSuccess;
        if (!b->exec) e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            b->captured.clear();
            return to_status(e);
        }
        b->captured.assign(probs, probs + count);
    }
    b->launches += b->graph_launches;
    return to_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

cv_status cv_batch_plan_options(cv_batch_t b, int32_t index, cv_plan_options *opts) {
    if (!b || !opts || index < 0 || index >= (int32_t)b->plans.size()) return CV_ERR_INVALID_ARG;
    *opts = b->opts[index];
    return CV_OK;
}

cv_status cv_batch_launches(cv_batch_t b, int64_t *count, int32_t *batched) {
    if (!b || !count) return CV_ERR_INVALID_ARG;
    *count = b->launches;
    if (batched) *batched = b->fused ? 1 : 0;
    return CV_OK;
}

cv_status cv_batch_status(cv_batch_t b, void *stream) {
    if (!b) return CV_ERR_INVALID_ARG;
    cv_status first = CV_OK;
    for (cv_plan_t p : b->plans) {
        const cv_status st = cv_plan_status(p, stream);
        if (first == CV_OK) first = st;
    }
    return first;
}

cv_status cv_batch_destroy(cv_batch_t b) {
    if (!b) return CV_OK;
    release(b);
    return CV_OK;
}

cv_status cv_products_batched(const cv_problem *probs, int32_t count, cv_dtype in_dtype, cv_dtype out_dtype,
                              cv_precision prec, void *stream) {
    cv_batch_t b = nullptr;
    cv_status st = cv_batch_plan(&b, probs, count, 1, in_dtype, out_dtype, prec, stream);
    if (st != CV_OK) return st;
    st = cv_batch_products(b, probs, stream);
    const cv_status dev = cv_batch_status(b, stream);
    if (st == CV_OK) st = dev;
    cv_batch_destroy(b);
    return st;
}

}  // extern "C"
