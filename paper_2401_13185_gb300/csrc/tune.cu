// tune.cu -- measured choice of plan options per problem shape:
// cv_tune_key, cv_tune_cache_get / cv_tune_cache_put (a JSON file) and
// cv_plan_tune.
//
// The options that change how the work is cut are the strategy (per-fold
// tiles that store each fold's Gram partials, or the small-fold strategy
// that recomputes each fold's part from its rows in the epilogue) and ctas
// (the number of contraction CTAs the segment lengths are tuned for: longer
// segments mean fewer partial tiles to write and reduce, shorter ones a
// better balanced contraction).  cv_plan's rule picks a strategy from the
// mean fold size and every SM for ctas; the tuner times the alternatives on
// the caller's data and keeps the fastest, keyed by the device and the
// problem's shape class, so that later plans of the same class can take the
// cached options without measuring.
#include <ctype.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "cvx_internal.cuh"

namespace {

struct TuneEntry {
    int strategy = 0, ctas = 0;
    double ms = 0.0;
};

int floor_log2(int64_t x) {
    int e = 0;
    while (x > 1) {
        x >>= 1;
        ++e;
    }
    return e;
}

const char *cache_path_of(const char *path) { return path ? path : getenv("CVX_TUNE_CACHE"); }

// Keys are written without JSON escapes, so they keep to this alphabet.
bool key_ok(const char *key) {
    if (!key || !*key) return false;
    for (const char *c = key; *c; ++c)
        if (!(isalnum((unsigned char)*c) || strchr("/^_.-", *c))) return false;
    return true;
}

// A small reader of the cache's one shape of JSON: an object of objects with
// the fields strategy, ctas and ms.  Entries are taken in order while the
// text parses; at the first malformed entry the rest is dropped.
struct Reader {
    const std::string &t;
    size_t i = 0;
    explicit Reader(const std::string &text) : t(text) {}
    void ws() {
        while (i < t.size() && isspace((unsigned char)t[i])) ++i;
    }
    bool eat(char c) {
        ws();
        if (i < t.size() && t[i] == c) {
            ++i;
            return true;
        }
        return false;
    }
    bool str(std::string &out) {
        if (!eat('"')) return false;
        const size_t j = t.find('"', i);
        if (j == std::string::npos) return false;
        out = t.substr(i, j - i);
        i = j + 1;
        return true;
    }
    bool num(double &out) {
        ws();
        const char *b = t.c_str() + i;
        char *e = nullptr;
        out = strtod(b, &e);
        if (e == b) return false;
        i += (size_t)(e - b);
        return true;
    }
};

void parse_cache(const std::string &text, std::map<std::string, TuneEntry> &out) {
    Reader r(text);
    if (!r.eat('{')) return;
    if (r.eat('}')) return;
    while (true) {
        std::string key;
        if (!r.str(key) || !r.eat(':') || !r.eat('{')) return;
        TuneEntry en;
        int seen = 0;
        while (true) {
            std::string f;
            double v;
            if (!r.str(f) || !r.eat(':') || !r.num(v)) return;
            if (f == "strategy") en.strategy = (int)v, seen |= 1;
            else if (f == "ctas") en.ctas = (int)v, seen |= 2;
            else if (f == "ms") en.ms = v, seen |= 4;
            if (r.eat(',')) continue;
            if (r.eat('}')) break;
            return;
        }
        if (seen == 7 && key_ok(key.c_str()) && en.strategy >= CV_STRATEGY_AUTO &&
            en.strategy <= CV_STRATEGY_SMALL_FOLDS && en.ctas >= 0 && en.ms >= 0.0)
            out[key] = en;
        if (r.eat(',')) continue;
        return;   // '}' or malformed: done either way
    }
}

bool read_file(const char *path, std::string &text) {
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
    fclose(f);
    return true;
}

bool write_cache(const char *path, const std::map<std::string, TuneEntry> &m) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return false;
    fprintf(f, "{");
    bool first = true;
    for (const auto &kv : m) {
        fprintf(f, "%s\n \"%s\": {\"strategy\": %d, \"ctas\": %d, \"ms\": %.6g}", first ? "" : ",", kv.first.c_str(),
                kv.second.strategy, kv.second.ctas, kv.second.ms);
        first = false;
    }
    fprintf(f, "\n}\n");
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

// Device buffers of one candidate run, freed on scope exit.
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

}  // namespace

extern "C" {

cv_status cv_tune_key(int64_t N, int32_t K, int32_t M, int32_t P, cv_dtype in_dtype, cv_dtype out_dtype,
                      cv_precision prec, char *key, int32_t size) {
    if (!key || size < 1 || N < 2 || K < 1 || M < 0 || P < 2 || (int64_t)P > N) return CV_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CV_ERR_CUDA;
    const int n = snprintf(key, (size_t)size, "sm%d/prec%d/in%d/out%d/K%d/M%d/N2^%d/rows2^%d", sms, (int)prec,
                           (int)in_dtype, (int)out_dtype, K, M, floor_log2(N), floor_log2(N / P));
    return n < 0 || n >= size ? CV_ERR_INVALID_ARG : CV_OK;
}

cv_status cv_tune_cache_get(const char *path, const char *key, cv_plan_options *opts, double *ms) {
    if (!key_ok(key) || !opts) return CV_ERR_INVALID_ARG;
    const char *file = cache_path_of(path);
    std::string text;
    if (!file || !read_file(file, text)) return CV_ERR_UNSUPPORTED;
    std::map<std::string, TuneEntry> m;
    parse_cache(text, m);
    const auto it = m.find(key);
    if (it == m.end()) return CV_ERR_UNSUPPORTED;
    *opts = cv_plan_options{};
    opts->strategy = it->second.strategy;
    opts->ctas = it->second.ctas;
    if (ms) *ms = it->second.ms;
    return CV_OK;
}

cv_status cv_tune_cache_put(const char *path, const char *key, const cv_plan_options *opts, double ms) {
    if (!key_ok(key) || !opts || opts->strategy < CV_STRATEGY_AUTO || opts->strategy > CV_STRATEGY_SMALL_FOLDS ||
        opts->ctas < 0 || !(ms >= 0.0))
        return CV_ERR_INVALID_ARG;
    const char *file = cache_path_of(path);
    if (!file) return CV_OK;
    std::map<std::string, TuneEntry> m;
    std::string text;
    if (read_file(file, text)) parse_cache(text, m);
    m[key] = TuneEntry{opts->strategy, opts->ctas, ms};
    return write_cache(file, m) ? CV_OK : CV_ERR_INVALID_ARG;
}

cv_status cv_plan_tune(int64_t N, int32_t K, int32_t M, int32_t P, const int32_t *fold_ids, int fold_ids_on_device,
                       cv_dtype in_dtype, cv_dtype out_dtype, cv_precision prec, const void *X, int64_t ldx,
                       const void *Y, int64_t ldy, int flags, int ddof, const char *cache_path,
                       cv_plan_options *best, double *best_ms, void *stream) {
    if (!best || !X || !fold_ids || (M > 0 && !Y)) return CV_ERR_INVALID_ARG;
    char key[160];
    cv_status s = cv_tune_key(N, K, M, P, in_dtype, out_dtype, prec, key, (int32_t)sizeof key);
    if (s != CV_OK) return s;
    const char *file = cache_path_of(cache_path);
    if (file && cv_tune_cache_get(file, key, best, best_ms) == CV_OK) return CV_OK;

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CV_ERR_CUDA;
    std::vector<cv_plan_options> cands;
    auto add = [&](int strategy, int ctas) {
        cv_plan_options o{};
        o.strategy = strategy;
        o.ctas = ctas;
        cands.push_back(o);
    };
    add(CV_STRATEGY_AUTO, 0);
    add(CV_STRATEGY_FOLD_GROUPED, std::max(1, sms / 2));
    if (N <= (int64_t)256 * P) {   // folds of at most 256 rows: both strategies are worth a try
        add(CV_STRATEGY_FOLD_GROUPED, 0);
        add(CV_STRATEGY_SMALL_FOLDS, 0);
    }

    const size_t el = out_dtype == CV_F64 ? sizeof(double) : sizeof(float);
    DevBuf xtx, xty, mean, sd;
    if (cudaMalloc(&xtx.p, el * (size_t)P * K * K) != cudaSuccess ||
        (M > 0 && cudaMalloc(&xty.p, el * (size_t)P * K * M) != cudaSuccess) ||
        cudaMalloc(&mean.p, sizeof(double) * (size_t)P * (K + M)) != cudaSuccess ||
        cudaMalloc(&sd.p, sizeof(double) * (size_t)P * (K + M)) != cudaSuccess) {
        cudaGetLastError();
        return CV_ERR_ALLOC;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return CV_ERR_CUDA;
    }
    double best_t = -1.0;
    cv_status first_err = CV_OK;
    for (size_t c = 0; c < cands.size(); ++c) {
        cv_plan_t pl = nullptr;
        s = cv_plan_ex(&pl, N, K, M, P, fold_ids, fold_ids_on_device, in_dtype, out_dtype, prec, &cands[c], stream);
        auto run = [&]() {
            return cv_products(pl, X, ldx, Y, ldy, flags, ddof, xtx.p, xty.p, (double *)mean.p, (double *)sd.p,
                               stream);
        };
        for (int w = 0; w < 2 && s == CV_OK; ++w) s = run();   // warm-up
        if (s == CV_OK) s = cudaStreamSynchronize(st) == cudaSuccess ? cv_plan_status(pl, stream) : CV_ERR_CUDA;
        double t = 0.0;
        if (s == CV_OK) {
            // at least 3 calls and about 20 ms of them
            int reps = 3, done = 0;
            float ms_all = 0.0f;
            while (s == CV_OK && done < 64) {
                cudaEventRecord(e0, st);
                for (int r = 0; r < reps && s == CV_OK; ++r) s = run();
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) s = CV_ERR_CUDA;
                float ms = 0.0f;
                if (s == CV_OK) cudaEventElapsedTime(&ms, e0, e1);
                ms_all += ms;
                done += reps;
                if (ms_all >= 20.0f) break;
                reps *= 2;
            }
            if (s == CV_OK) s = cv_plan_status(pl, stream);
            t = ms_all / done;
        }
        if (pl) cv_plan_destroy(pl);
        if (s != CV_OK) {
            if (first_err == CV_OK) first_err = s;
            if (s == CV_ERR_CUDA) break;   // the device is in trouble: stop measuring
            continue;                      // a candidate this problem does not support
        }
        if (best_t < 0.0 || t < best_t) {
            best_t = t;
            *best = cands[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_t < 0.0) return first_err != CV_OK ? first_err : CV_ERR_UNSUPPORTED;
    if (best_ms) *best_ms = best_t;
    if (file) cv_tune_cache_put(file, key, best, best_t);
    return CV_OK;
}

}  // extern "C"
