// Autotuner of the engine settings (gumap_knn_autotune) and its cache.
//
// Settings are timed on the handle's own graph through the public calls
// (gumap_knn_set_option, gumap_knn_run): for the full form the MS-BFS state
// budget (it sets the source-block width), the pull item width, the degree
// multiplier above which a vertex's items are warp-wide, then on the best of
// those the CTAs per SM (the CTA shape), the staging of rows in shared
// memory and the automatic level direction at three push thresholds; for the
// partial form the engine and the frontier engine's merge (one thread or
// one warp per source); for single graphs that fit a CTA's shared memory
// also the batched engine with four unit widths; for batch handles the
// widest unit (the
// source-block width of the batched engine). Each candidate runs once to
// warm up, then three times with the L2 flushed before each run; the median
// device time decides. The winner is kept in a JSON-lines cache under a key
// of the graph's shape class, so graphs of the same class start tuned.
#include "gumap.h"
#include "gumap_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <string>
#include <vector>

namespace {

struct Setting {
    int engine = GUMAP_ENGINE_AUTO;
    int pull_width = 4;
    int heavy_mult = 4;
    int direction = 1;
    long long state_bytes = 0;
    int ctas_per_sm = 3;
    int stage = 1;
    int push_div = 8;
    int batch_width = 0;  // batch handles only
    int frontier_build = 0;  // partial form, frontier engine
};

std::string shape_key(const gumap_knn_info& in) {
    const double mean = in.n > 0 ? (double)in.nnz / in.n : 0.0;
    const double hub = in.max_degree / std::max(mean, 1.0);
    char buf[160];
    snprintf(buf, sizeof(buf), "%s/k%d/w%d/logn%.2f/logdeg%.1f/loghub%d", in.mode == GUMAP_FULL ? "full" : "partial",
             in.k, (in.flags & GUMAP_WEIGHTS_DIRECTED) ? 0 : 1, std::round(std::log2((double)in.n) * 4.0) / 4.0,
             std::round(std::log2(mean + 1.0) * 2.0) / 2.0, (int)std::lround(std::log2(hub + 1.0)));
    return buf;
}

bool read_cache(const char* path, const std::string& key, Setting* s) {
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        char k[200];
        Setting t;
        double ms = 0;
        if (sscanf(line.c_str(),
                   "{\"key\": \"%199[^\"]\", \"engine\": %d, \"pull_width\": %d, \"heavy_mult\": %d, "
                   "\"direction\": %d, \"state_bytes\": %lld, \"ctas_per_sm\": %d, \"stage\": %d, "
                   "\"push_div\": %d, \"frontier_build\": %d, \"batch_width\": %d, \"ms\": %lf}",
                   k, &t.engine, &t.pull_width, &t.heavy_mult, &t.direction, &t.state_bytes, &t.ctas_per_sm,
                   &t.stage, &t.push_div, &t.frontier_build, &t.batch_width, &ms) == 12 &&
            key == k) {
            *s = t;  // the last entry of a key wins
            found = true;
        }
    }
    return found;
}

void append_cache(const char* path, const std::string& key, const Setting& s, double ms) {
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{\"key\": \"%s\", \"engine\": %d, \"pull_width\": %d, \"heavy_mult\": %d, \"direction\": %d, "
            "\"state_bytes\": %lld, \"ctas_per_sm\": %d, \"stage\": %d, \"push_div\": %d, "
            "\"frontier_build\": %d, \"batch_width\": %d, \"ms\": %.6f}\n",
            key.c_str(), s.engine, s.pull_width, s.heavy_mult, s.direction, s.state_bytes, s.ctas_per_sm, s.stage,
            s.push_div, s.frontier_build, s.batch_width, ms);
    fclose(f);
}

int apply(gumap_knn* h, const gumap_knn_info& in, const Setting& s) {
    int rc;
    if (in.batch) return gumap_knn_set_option(h, GUMAP_OPT_BATCH_WIDTH, s.batch_width);
    if ((rc = gumap_knn_set_option(h, GUMAP_OPT_ENGINE, s.engine))) return rc;
    if (s.engine == GUMAP_ENGINE_BATCH) return gumap_knn_set_option(h, GUMAP_OPT_BATCH_WIDTH, s.batch_width);
    if (s.engine == GUMAP_ENGINE_FRONTIER &&
        (rc = gumap_knn_set_option(h, GUMAP_OPT_FRONTIER_BUILD, s.frontier_build)))
        return rc;
    if (s.engine == GUMAP_ENGINE_MSBFS || s.engine == GUMAP_ENGINE_AUTO) {
        const long long mean = in.n > 0 ? in.nnz / in.n : 0;
        if ((rc = gumap_knn_set_option(h, GUMAP_OPT_STATE_BYTES, s.state_bytes))) return rc;
        if ((rc = gumap_knn_set_option(h, GUMAP_OPT_PULL_WIDTH, s.pull_width))) return rc;
        if ((rc = gumap_knn_set_option(h, GUMAP_OPT_DIRECTION, s.direction))) return rc;
        if ((rc = gumap_knn_set_option(h, GUMAP_OPT_CTAS_PER_SM, s.ctas_per_sm))) return rc;
        if ((rc = gumap_knn_set_option(h, GUMAP_OPT_STAGE, s.stage))) return rc;
        if ((rc = gumap_knn_set_option(h, GUMAP_OPT_PUSH_DIV, s.push_div))) return rc;
        if ((rc = gumap_knn_set_option(h, GUMAP_OPT_HEAVY_DEGREE, std::max<long long>(64, s.heavy_mult * mean))))
            return rc;
    }
    return GUMAP_OK;
}

// A single graph small enough for one CTA's shared memory may run on the
// batched engine (a level costs a __syncthreads instead of a grid barrier):
// units of 32, 8, 2 and 1 words.
void add_batch_candidates(const gumap_knn_info& in, std::vector<Setting>& cands) {
    if (in.batch || in.n > 27000) return;
    for (int w : {32, 8, 2, 1}) {
        Setting s;
        s.engine = GUMAP_ENGINE_BATCH;
        s.batch_width = w;
        cands.push_back(s);
    }
}

}  // namespace

namespace gumap {

// Applies cached settings at handle creation (GUMAP_TUNE_CACHE); silent on
// any failure: the handle keeps its defaults.
void tune_apply_cached(gumap_knn* h, const char* path) {
    gumap_knn_info in;
    if (!path || !*path || gumap_knn_get_info(h, &in) != GUMAP_OK || in.batch) return;
    Setting s;
    if (read_cache(path, shape_key(in), &s)) apply(h, in, s);
}

}  // namespace gumap

extern "C" int gumap_knn_autotune(gumap_knn* h, const char* cache_path, gumap_tune_result* out) {
    gumap_knn_info in;
    int rc = gumap_knn_get_info(h, &in);
    if (rc) return rc;
    gumap_tune_result res;
    std::memset(&res, 0, sizeof(res));
    const std::string key = shape_key(in);
    Setting best;
    if (!in.batch && cache_path && read_cache(cache_path, key, &best)) {
        if ((rc = apply(h, in, best))) return rc;
        res.from_cache = 1;
        res.engine = best.engine;
        res.pull_width = best.pull_width;
        res.heavy_mult = best.heavy_mult;
        res.direction = best.direction;
        res.state_bytes = best.state_bytes;
        res.ctas_per_sm = best.ctas_per_sm;
        res.stage = best.stage;
        res.push_div = best.push_div;
        res.frontier_build = best.frontier_build;
        if (out) *out = res;
        return GUMAP_OK;
    }

    const size_t cells = (size_t)in.n * in.k;
    void *idx = nullptr, *dist = nullptr, *w = nullptr, *flush = nullptr;
    const size_t flush_bytes = 256ull << 20;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (st) cudaStreamSynchronize(st);
        cudaFree(idx);
        cudaFree(dist);
        cudaFree(w);
        cudaFree(flush);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
    };
    if (cudaMalloc(&idx, cells * 4) != cudaSuccess || cudaMalloc(&dist, cells * 2) != cudaSuccess ||
        cudaMalloc(&w, cells * 4) != cudaSuccess || cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        cleanup();
        return GUMAP_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return GUMAP_ERR_CUDA;
    }
    // median device time of three runs (L2 flushed before each), after one warm-up run
    auto time_run = [&](double* ms) -> int {
        int r = gumap_knn_run(h, nullptr, in.n, (int32_t*)idx, (uint16_t*)dist, (float*)w, st);
        if (r) return r;
        double t[3];
        for (int i = 0; i < 3; ++i) {
            if (cudaMemsetAsync(flush, i, flush_bytes, st) != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess)
                return GUMAP_ERR_CUDA;
            if ((r = gumap_knn_run(h, nullptr, in.n, (int32_t*)idx, (uint16_t*)dist, (float*)w, st))) return r;
            float f = 0.0f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&f, e0, e1) != cudaSuccess)
                return GUMAP_ERR_CUDA;
            t[i] = f;
        }
        std::sort(t, t + 3);
        *ms = t[1];
        return gumap_knn_check(h, st);
    };

    std::vector<Setting> cands;
    if (in.batch) {  // the widest unit: wide units share each level's sweep, narrow ones balance the CTAs
        for (int w : {64, 32, 16, 8}) {
            Setting s;
            s.batch_width = w;
            cands.push_back(s);
        }
    } else if (in.mode == GUMAP_FULL) {
        add_batch_candidates(in, cands);
        for (long long budget : {96ll << 20, 256ll << 20, 1024ll << 20})
            for (int width : {4, 2})
                for (int hm : {2, 4, 8}) {
                    Setting s;
                    s.engine = GUMAP_ENGINE_MSBFS;
                    s.state_bytes = budget;
                    s.pull_width = width;
                    s.heavy_mult = hm;
                    s.direction = 1;
                    cands.push_back(s);
                }
    } else {
        add_batch_candidates(in, cands);
        // the frontier engine's merges (a group of lanes, one thread or one warp per source)
        for (int b : {3, 1, 2}) {
            if (b == 1 && in.k > 64) continue;  // the thread build covers k <= 64
            Setting f;
            f.engine = GUMAP_ENGINE_FRONTIER;
            f.frontier_build = b;
            cands.push_back(f);
        }
        // The MS-BFS engine sweeps the bitsets of all n vertices at every
        // level of every source block: at least 3 n^2 / 8 bytes per level
        // over all blocks. Beyond 64 GB of that (n above about 400,000) one
        // timing run would take seconds against the frontier engine's
        // milliseconds, so it is not a candidate there.
        if (3.0 * (double)in.n * (double)in.n / 8.0 <= 64e9)
            for (long long budget : {96ll << 20, 256ll << 20}) {
                Setting s;
                s.engine = GUMAP_ENGINE_MSBFS;
                s.state_bytes = budget;
                cands.push_back(s);
            }
    }
    double default_ms = 0.0;
    if ((rc = time_run(&default_ms))) {
        cleanup();
        return rc;
    }
    double best_ms = 1e300;
    for (const Setting& s : cands) {
        double ms = 0.0;
        rc = apply(h, in, s);
        if (rc == GUMAP_ERR_TOO_LARGE && s.engine == GUMAP_ENGINE_BATCH) continue;  // the graph does not fit a CTA
        if (rc || (rc = time_run(&ms))) {
            cleanup();
            return rc;
        }
        res.candidates++;
        if (ms < best_ms) {
            best_ms = ms;
            best = s;
        }
    }
    if (!in.batch && in.mode == GUMAP_FULL) {
        // then, one at a time on the best so far: CTA shape, staging, and the
        // automatic direction at three push thresholds
        for (int step = 0; step < 5; ++step) {
            Setting s = best;
            if (step == 0) s.ctas_per_sm = best.ctas_per_sm == 4 ? 3 : 4;
            else if (step == 1) s.stage = best.stage ? 0 : 1;
            else {
                s.direction = 0;
                s.push_div = step == 2 ? 8 : step == 3 ? 64 : 512;
            }
            double ms = 0.0;
            if ((rc = apply(h, in, s)) || (rc = time_run(&ms))) {
                cleanup();
                return rc;
            }
            res.candidates++;
            if (ms < best_ms) {
                best_ms = ms;
                best = s;
            }
        }
    }
    cleanup();
    if ((rc = apply(h, in, best))) return rc;
    if (cache_path && !in.batch) append_cache(cache_path, key, best, best_ms);
    res.best_ms = best_ms;
    res.default_ms = default_ms;
    res.engine = best.engine;
    res.pull_width = best.pull_width;
    res.heavy_mult = best.heavy_mult;
    res.direction = best.direction;
    res.state_bytes = best.state_bytes;
    res.ctas_per_sm = best.ctas_per_sm;
    res.stage = best.stage;
    res.push_div = best.push_div;
    res.batch_width = best.batch_width;
    res.frontier_build = best.frontier_build;
    if (out) *out = res;
    return GUMAP_OK;
}
