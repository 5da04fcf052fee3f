// batch.cu -- batches of independent cross-validation problems.
//
// Each problem keeps its own plan (Algorithm 1 and workspace).  The products
// of all problems are enqueued as one CUDA graph: a fork event on an internal
// origin stream, every problem's cv_products on one of up to 32 internal
// worker streams (in decreasing order of work, round-robin), and a join back to the
// origin.  The branches of the graph are independent, so the GPU overlaps the
// problems' kernels; one graph launch replaces hundreds of kernel launches.
// The graph is kept and relaunched while the problem descriptors stay the
// same; a changed descriptor (new buffers or flags) triggers a re-capture,
// applied as an in-place update of the executable graph when its topology
// allows.
#include <algorithm>
#include <new>
#include <vector>

#include "cvx_internal.cuh"

struct cv_batch_s {
    std::vector<cv_plan_t> plans;
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

}  // namespace

extern "C" {

cv_status cv_batch_plan(cv_batch_t *out, const cv_problem *probs, int32_t count, int fold_ids_on_device,
                        cv_dtype in_dtype, cv_dtype out_dtype, cv_precision prec, void *stream) {
    if (!out) return CV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!probs || count < 1) return CV_ERR_INVALID_ARG;
    cv_batch_s *b = new (std::nothrow) cv_batch_s();
    if (!b) return CV_ERR_ALLOC;
    for (int i = 0; i < count; ++i) {
        const cv_problem &q = probs[i];
        cv_plan_t p = nullptr;
        const cv_status st =
            cv_plan(&p, q.N, q.K, q.M, q.P, q.fold_ids, fold_ids_on_device, in_dtype, out_dtype, prec, stream);
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
    bool same = b->exec && b->captured.size() == (size_t)count;
    for (int i = 0; same && i < count; ++i) same = same_problem(b->captured[i], probs[i]);
    if (!same) {
        cudaGraph_t g = nullptr;
        const cv_status st = capture(b, probs, &g);
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
    return to_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
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
