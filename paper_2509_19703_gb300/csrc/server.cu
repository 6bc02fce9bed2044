// Request server: continuous batching of independent graph requests.
//
// One scheduler thread owns every CUDA call of the server. It admits waiting
// requests in arrival order while their device memory fits the budget (a
// single arena allocated at creation and sub-allocated first-fit, so serving
// never calls cudaMalloc or cudaFree), forms launches -- waiting small
// graphs of the same k together in one batched launch (batch.cu), a graph too
// large for it alone (frontier.cu for the partial form, msbfs.cu for the full
// form) -- and keeps up to n_streams launches in flight on separate streams,
// the last of which takes small-graph batches only. A large graph's launches
// are sized for half the SMs, so small batches keep running beside them.
// Each launch runs the whole path of gumap_knn_run without the COO: BFS kNN
// lists, rho/sigma and the weights (weights.cu), the fuzzy union, then ids made local to
// each request's graph. A host callback enqueued after the launch stamps its
// completion. Requests that arrive meanwhile wait only for a free stream and
// memory, so launches overlap on the device.
#include "gumap.h"
#include "gumap_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace gumap {

namespace {

__global__ void localize_kernel(int32_t* __restrict__ idx, long long rows, int k, const int32_t* __restrict__ offs,
                                int n_graphs) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_graphs;  // graph g with offs[g] <= r < offs[g + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (offs[mid] <= r) lo = mid;
            else hi = mid;
        }
        const int v0 = offs[lo];
        int32_t* row = idx + r * k;
        for (int t = 0; t < k; ++t)
            if (row[t] >= 0) row[t] -= v0;
    }
}

// First-fit allocator over [0, cap) with coalescing; 256-byte granules.
class RangeAllocator {
public:
    explicit RangeAllocator(size_t cap = 0) { reset(cap); }
    void reset(size_t cap) {
        free_.clear();
        cap_ = cap;
        used_ = 0;
        if (cap) free_[0] = cap;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = round(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t capacity() const { return cap_; }
    static size_t round(size_t b) { return (b + 255) / 256 * 256; }

private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0;
};

// Sequential carve-out of one allocation into typed sub-buffers.
struct Carver {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        const size_t at = off;
        off += RangeAllocator::round(count * sizeof(T));
        return at;
    }
};

struct Launch;

struct Request {
    uint64_t id = 0;
    int32_t n = 0, k = 0;
    int64_t nnz = 0;
    int mode = GUMAP_FULL;
    std::vector<int32_t> rp, col;  // host copy until uploaded
    int state = 0;                 // 0 waiting, 1 running, 2 done
    int status = GUMAP_PENDING;
    double t_submit = 0, t_start = 0, t_done = 0;
    Launch* launch = nullptr;
    long long row_off = 0;         // first row in the launch's outputs
    bool released = false;
};

struct Launch {
    std::vector<Request*> reqs;
    int stream = 0;
    int engine = 0;
    size_t arena_off = 0, arena_bytes = 0;
    size_t stage_off = 0, stage_bytes = 0;
    int32_t* idx = nullptr;
    uint16_t* dist = nullptr;
    float* w = nullptr;
    int32_t* status_host = nullptr;  // pinned word the launch copies its device status into
    std::atomic<int> done{0};
    double t_done = 0;
    bool finished = false;           // completion processed by the scheduler
    int n_released = 0;
    struct gumap_server* srv = nullptr;
};

}  // namespace

}  // namespace gumap

using namespace gumap;

struct gumap_server {
    int device = 0;
    gumap_server_opts opts{};
    int num_sms = 0;
    int coop_grid = 0;
    int batch_grid = 0;
    unsigned char* arena = nullptr;
    unsigned char* staging = nullptr;  // pinned host
    RangeAllocator arena_alloc, stage_alloc;
    size_t arena_peak = 0;
    std::vector<cudaStream_t> streams;
    std::vector<int> in_flight;        // launches per stream
    std::chrono::steady_clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> waiting;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<std::unique_ptr<Launch>> launches;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    int64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_released = 0, n_launches = 0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

constexpr int kBatchMaxN = 27000;  // graphs above this run alone (they do not fit a CTA's shared memory)

void CUDART_CB launch_done(void* p) {
    Launch* L = static_cast<Launch*>(p);
    gumap_server* srv = L->srv;  // L may be freed as soon as `done` is set
    L->t_done = srv->now();
    L->done.store(1);
    srv->cv.notify_all();
}

bool is_small(const Request* r) { return r->n <= kBatchMaxN; }

// Device bytes of the per-row outputs and weight scratch.
size_t rows_bytes(long long rows, int k) {
    return RangeAllocator::round((size_t)rows * k * 4) * 3 + RangeAllocator::round((size_t)rows * k * 2) +
           2 * RangeAllocator::round((size_t)rows * 4);
}

// Device bytes a request needs when it runs alone as a large graph.
size_t alone_bytes(const gumap_server* s, const Request* r) {
    size_t b = 4096 + RangeAllocator::round(((size_t)r->n + 1) * 4) + RangeAllocator::round((size_t)r->nnz * 4) +
               rows_bytes(r->n, r->k);
    if (r->mode == GUMAP_FULL) {
        const size_t W = 4;  // the narrowest block (128 sources) bounds the bitsets from below
        b += 3 * RangeAllocator::round((size_t)r->n * W * 4) + RangeAllocator::round((size_t)r->n * 4) + 4096;
    }
    (void)s;
    return b;
}

// Launch one set of requests. Called by the scheduler with the lock held.
// Returns false if memory is short (nothing launched, nothing changed).
bool start_launch(gumap_server* s, std::vector<Request*>& group, int stream) {
    const int k = group[0]->k;
    const bool small = is_small(group[0]);
    const bool want_union = !(s->opts.flags & GUMAP_WEIGHTS_DIRECTED);
    const int ng = (int)group.size();
    std::vector<int32_t> offs(ng + 1, 0);
    long long nnz = 0;
    for (int g = 0; g < ng; ++g) {
        offs[g + 1] = offs[g] + group[g]->n;
        nnz += group[g]->nnz;
    }
    const long long N = offs[ng];

    // plan
    std::vector<BatchUnit> units;
    size_t smem = 0;
    long long slab = 0;
    std::vector<int32_t> rp_union;
    std::vector<int32_t> modes(ng);
    for (int g = 0; g < ng; ++g) modes[g] = group[g]->mode;
    rp_union.resize((size_t)N + 1);
    {
        long long e = 0;
        for (int g = 0; g < ng; ++g) {
            const Request* r = group[g];
            for (int32_t v = 0; v < r->n; ++v) rp_union[(size_t)offs[g] + v] = (int32_t)(e + r->rp[(size_t)v]);
            e += r->nnz;
        }
        rp_union[(size_t)N] = (int32_t)e;
    }
    int W = 0, nblocks = 0;  // full form of a large graph: MS-BFS blocks
    if (small) {
        std::vector<int64_t> edges((size_t)ng);
        for (int g = 0; g < ng; ++g) edges[(size_t)g] = group[g]->nnz;
        if (plan_batch(ng, offs.data(), edges.data(), modes.data(), units, smem, slab) >= 0) return false;
    } else if (group[0]->mode == GUMAP_FULL) {
        const double budget = 96.0 * 1024 * 1024;
        long long S = (long long)(budget * 8.0 / (3.0 * (double)N)) / 128 * 128;
        if (S < 128) S = 128;
        if (S > 32768) S = 32768;
        nblocks = (int)((N + S - 1) / S);
        S = ((N + nblocks - 1) / nblocks + 127) / 128 * 128;
        W = (int)(S / 32);
    }

    // device layout
    Carver c;
    const size_t o_ctr = c.take<DeviceCounters>(1);
    const size_t o_rp = c.take<int32_t>((size_t)N + 1);
    const size_t o_col = c.take<int32_t>((size_t)std::max<long long>(nnz, 1));
    const size_t o_offs = c.take<int32_t>((size_t)ng + 1);
    const size_t o_units = c.take<BatchUnit>(std::max<size_t>(units.size(), 1));
    const size_t o_idx = c.take<int32_t>((size_t)N * k);
    const size_t o_dist = c.take<uint16_t>((size_t)N * k);
    const size_t o_w = c.take<float>((size_t)N * k);
    const size_t o_rec = c.take<WeightRow>((size_t)N);
    const size_t o_rho = c.take<float>((size_t)N);
    const size_t o_sigma = c.take<float>((size_t)N);
    size_t o_slab = 0, o_bits = 0, o_act = 0, o_need = 0, o_cnt = 0, o_order = 0, o_queue = 0;
    if (small && slab > 0) o_slab = c.take<uint32_t>((size_t)slab * s->batch_grid);
    if (!small && group[0]->mode == GUMAP_FULL) {
        o_bits = c.take<uint32_t>((size_t)N * W * 3);
        o_act = c.take<uint32_t>((size_t)W);
        o_need = c.take<uint32_t>((size_t)W);
        o_cnt = c.take<int32_t>((size_t)W * 32);
        o_order = c.take<int32_t>((size_t)N);
        o_queue = c.take<int32_t>((size_t)N * 5);  // 4 frontier queues + queue-entry levels
    }
    const size_t dev_bytes = c.off;
    // pinned staging: status word, rp, col, offs, units
    Carver h;
    const size_t h_status = h.take<int32_t>(1);
    const size_t h_rp = h.take<int32_t>((size_t)N + 1);
    const size_t h_col = h.take<int32_t>((size_t)std::max<long long>(nnz, 1));
    const size_t h_offs = h.take<int32_t>((size_t)ng + 1);
    const size_t h_units = h.take<BatchUnit>(std::max<size_t>(units.size(), 1));
    const size_t stage_bytes = h.off;

    size_t aoff = 0, soff = 0;
    if (!s->arena_alloc.alloc(dev_bytes, &aoff)) return false;
    if (!s->stage_alloc.alloc(stage_bytes, &soff)) {
        s->arena_alloc.release(aoff, dev_bytes);
        return false;
    }
    s->arena_peak = std::max(s->arena_peak, s->arena_alloc.used());
    unsigned char* D = s->arena + aoff;
    unsigned char* H = s->staging + soff;
    auto dptr = [&](size_t o) { return D + o; };

    // stage the union CSR with ids shifted to the launch's numbering
    std::memcpy(H + h_rp, rp_union.data(), ((size_t)N + 1) * 4);
    {
        int32_t* col = reinterpret_cast<int32_t*>(H + h_col);
        long long e = 0;
        for (int g = 0; g < ng; ++g) {
            const Request* r = group[g];
            const int32_t sh = offs[g];
            for (long long q = 0; q < r->nnz; ++q) col[e + q] = r->col[(size_t)q] + sh;
            e += r->nnz;
        }
    }
    std::memcpy(H + h_offs, offs.data(), ((size_t)ng + 1) * 4);
    if (!units.empty()) std::memcpy(H + h_units, units.data(), units.size() * sizeof(BatchUnit));
    *reinterpret_cast<int32_t*>(H + h_status) = GUMAP_PENDING;

    cudaStream_t st = s->streams[stream];
    auto L = std::make_unique<Launch>();
    L->srv = s;
    L->stream = stream;
    L->arena_off = aoff;
    L->arena_bytes = dev_bytes;
    L->stage_off = soff;
    L->stage_bytes = stage_bytes;
    L->idx = reinterpret_cast<int32_t*>(dptr(o_idx));
    L->dist = reinterpret_cast<uint16_t*>(dptr(o_dist));
    L->w = reinterpret_cast<float*>(dptr(o_w));
    L->status_host = reinterpret_cast<int32_t*>(H + h_status);
    DeviceCounters* ctr = reinterpret_cast<DeviceCounters*>(dptr(o_ctr));
    int32_t* d_rp = reinterpret_cast<int32_t*>(dptr(o_rp));
    int32_t* d_col = reinterpret_cast<int32_t*>(dptr(o_col));
    int32_t* d_offs = reinterpret_cast<int32_t*>(dptr(o_offs));
    WeightRow* d_rec = reinterpret_cast<WeightRow*>(dptr(o_rec));

    bool ok = true;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess) ok = false;
    };
    ck(cudaMemcpyAsync(d_rp, H + h_rp, ((size_t)N + 1) * 4, cudaMemcpyHostToDevice, st));
    if (nnz > 0) ck(cudaMemcpyAsync(d_col, H + h_col, (size_t)nnz * 4, cudaMemcpyHostToDevice, st));
    ck(cudaMemcpyAsync(d_offs, H + h_offs, ((size_t)ng + 1) * 4, cudaMemcpyHostToDevice, st));
    ck(cudaMemsetAsync(ctr, 0, sizeof(DeviceCounters), st));
    if (small) {
        ck(cudaMemcpyAsync(dptr(o_units), H + h_units, units.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice, st));
        BatchArgs a{};
        a.row_ptr = d_rp;
        a.col = d_col;
        a.units = reinterpret_cast<BatchUnit*>(dptr(o_units));
        a.n_units = (int32_t)units.size();
        a.k = k;
        a.out_idx = L->idx;
        a.out_dist = L->dist;
        a.vslab = slab > 0 ? reinterpret_cast<uint32_t*>(dptr(o_slab)) : nullptr;
        a.vslab_words = slab;
        a.next_unit = &ctr->aux_count;
        a.ctr = ctr;
        ck(launch_batch(a, s->batch_grid, smem, st));
        L->engine = GUMAP_ENGINE_BATCH;
    } else if (group[0]->mode == GUMAP_PARTIAL) {
        FrontierArgs a{};
        a.row_ptr = d_rp;
        a.col = d_col;
        a.n = (int32_t)N;
        a.src = nullptr;
        a.n_src = (int32_t)N;
        a.k = k;
        a.out_idx = L->idx;
        a.out_dist = L->dist;
        a.status = &ctr->status;
        a.sms = (s->num_sms + 1) / 2;  // a large graph fills half the GPU: batches of small ones keep the rest
        ck(launch_frontier(a, st));
        L->engine = GUMAP_ENGINE_FRONTIER;
    } else {
        uint32_t* bits = reinterpret_cast<uint32_t*>(dptr(o_bits));
        int32_t* order = reinterpret_cast<int32_t*>(dptr(o_order));
        ck(launch_identity(order, (int32_t)N, st));
        const size_t words = (size_t)N * W;
        const int S = 32 * W;
        for (int b = 0; b < nblocks; ++b) {
            MsbfsArgs a{};
            a.row_ptr = d_rp;
            a.col = d_col;
            a.n = (int32_t)N;
            a.src = order + (size_t)b * S;
            a.identity = 1;  // order holds 0 .. N-1
            a.src_lo = b * S;
            a.nb = (int32_t)std::min<long long>(S, N - (long long)b * S);
            a.W = W;
            a.F = bits;
            a.N = bits + words;
            a.S = bits + 2 * words;
            a.heavy = order;
            a.n_heavy = 0;
            a.light = order;
            a.n_light = (int32_t)N;
            a.act = reinterpret_cast<uint32_t*>(dptr(o_act));
            a.need = reinterpret_cast<uint32_t*>(dptr(o_need));
            a.cnt = reinterpret_cast<int32_t*>(dptr(o_cnt));
            a.out_idx = L->idx + (size_t)b * S * k;
            a.out_dist = L->dist + (size_t)b * S * k;
            a.k = k;
            a.partial = 0;
            a.ctr = ctr;
            a.direction = 1;  // pull only (see GUMAP_OPT_DIRECTION)
            a.seen_only = 1;  // so the levels pull from the seen sets (MsbfsArgs::seen_only)
            a.push_div = 8;
            a.queue = reinterpret_cast<int32_t*>(dptr(o_queue));
            a.inq = a.queue + 4 * (size_t)N;
            ck(cudaMemsetAsync(ctr, 0, kLaunchCounterBytes, st));
            // half the resident grid: a large graph's hundreds of levels never hold the whole GPU
            ck(launch_msbfs(a, msbfs_grid_for(a, std::max(1, s->coop_grid / 2)), 256, st));
        }
        L->engine = GUMAP_ENGINE_MSBFS;
    }
    const float T = (float)std::log2((double)k);
    float* rho = reinterpret_cast<float*>(dptr(o_rho));
    float* sigma = reinterpret_cast<float*>(dptr(o_sigma));
    ck(launch_smooth_knn(L->idx, L->dist, (int32_t)N, k, T, rho, sigma, want_union ? d_rec : nullptr,
                         want_union ? nullptr : L->w, st));
    if (want_union)
        ck(launch_union(L->idx, L->dist, d_rec, (int32_t)N, k, L->w, st));
    if (ng > 1) {
        long long grid = (N + 255) / 256;
        if (grid > 4096) grid = 4096;
        localize_kernel<<<(unsigned)grid, 256, 0, st>>>(L->idx, N, k, d_offs, ng);
        ck(cudaGetLastError());
    }
    ck(cudaMemcpyAsync(L->status_host, &ctr->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    ck(cudaLaunchHostFunc(st, launch_done, L.get()));
    if (!ok) {
        // launching failed: nothing will complete; fail the requests now
        cudaStreamSynchronize(st);
        for (Request* r : group) {
            r->state = 2;
            r->status = GUMAP_ERR_CUDA;
            r->t_done = s->now();
            s->n_failed++;
        }
        s->arena_alloc.release(aoff, dev_bytes);
        s->stage_alloc.release(soff, stage_bytes);
        return true;
    }
    const double t = s->now();
    for (int g = 0; g < ng; ++g) {
        Request* r = group[g];
        r->state = 1;
        r->t_start = t;
        r->launch = L.get();
        r->row_off = offs[g];
        L->reqs.push_back(r);
        std::vector<int32_t>().swap(r->rp);  // staged: the host copy is no longer needed
        std::vector<int32_t>().swap(r->col);
    }
    s->in_flight[stream]++;
    s->n_launches++;
    s->launches.push_back(std::move(L));
    return true;
}

void free_launch_if_released(gumap_server* s, Launch* L) {
    if (!L->finished || L->n_released < (int)L->reqs.size()) return;
    s->arena_alloc.release(L->arena_off, L->arena_bytes);
    for (Request* r : L->reqs) s->reqs.erase(r->id);
    for (auto it = s->launches.begin(); it != s->launches.end(); ++it)
        if (it->get() == L) {
            s->launches.erase(it);
            break;
        }
}

void scheduler(gumap_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // completions
        std::vector<Launch*> done_now;
        for (auto& L : s->launches)
            if (!L->finished && L->done.load()) done_now.push_back(L.get());
        for (Launch* L : done_now) {
            L->finished = true;
            s->in_flight[L->stream]--;
            s->stage_alloc.release(L->stage_off, L->stage_bytes);
            const int st = *L->status_host;
            for (Request* r : L->reqs) {
                r->state = 2;
                r->status = st == GUMAP_OK ? GUMAP_OK : st;
                r->t_done = L->t_done;
                if (st == GUMAP_OK) s->n_completed++;
                else s->n_failed++;
            }
            free_launch_if_released(s, L);
        }
        if (s->stop && s->launches.empty()) break;
        bool progress = !done_now.empty();
        // admission and launches
        while (!s->stop && !s->waiting.empty()) {
            // The last stream serves small graphs only, so large launches (a
            // full-form BFS over a large graph runs hundreds of levels) can never
            // hold every stream while small requests wait behind them.
            const int ns = (int)s->streams.size();
            int stream = -1, small_stream = -1;
            for (int i = 0; i < ns; ++i)
                if (s->in_flight[i] == 0) {
                    if (ns > 1 && i == ns - 1) small_stream = i;
                    else if (stream < 0) stream = i;
                }
            // the oldest waiting request that a free stream may take
            Request* r0 = nullptr;
            for (Request* r : s->waiting) {
                if (is_small(r) ? (stream >= 0 || small_stream >= 0) : stream >= 0) {
                    r0 = r;
                    break;
                }
            }
            if (!r0) break;
            if (is_small(r0) && stream < 0) stream = small_stream;
            std::vector<Request*> group{r0};
            if (is_small(r0)) {
                long long verts = r0->n;
                for (size_t i = 0; i < s->waiting.size() && (int)group.size() < s->opts.max_batch_graphs; ++i) {
                    Request* r = s->waiting[i];
                    if (r == r0 || r->k != r0->k || !is_small(r)) continue;
                    if (verts + r->n > s->opts.max_batch_vertices) break;
                    group.push_back(r);
                    verts += r->n;
                }
            }
            bool launched = start_launch(s, group, stream);
            while (!launched && group.size() > 1) {  // memory short: try a smaller group
                group.resize(group.size() / 2);
                launched = start_launch(s, group, stream);
            }
            if (!launched) {
                bool idle = s->arena_alloc.used() == 0;
                for (int f : s->in_flight) idle = idle && f == 0;
                if (!idle) break;  // wait for memory to be released
                // it does not fit an empty budget: it never will
                r0->state = 2;
                r0->status = GUMAP_ERR_TOO_LARGE;
                r0->t_done = s->now();
                s->n_failed++;
                s->waiting.erase(std::find(s->waiting.begin(), s->waiting.end(), r0));
                progress = true;
                continue;
            }
            for (Request* r : group) {
                auto it = std::find(s->waiting.begin(), s->waiting.end(), r);
                if (it != s->waiting.end()) s->waiting.erase(it);
            }
            progress = true;
        }
        if (!progress) s->cv.wait_for(lk, std::chrono::microseconds(200));
    }
}

}  // namespace

extern "C" {

int gumap_server_create(gumap_server** out, int device, uint64_t hbm_budget_bytes, const gumap_server_opts* opts) {
    if (!out) return GUMAP_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return GUMAP_ERR_CUDA;
    if (device < 0 || device >= ndev || hbm_budget_bytes < (1ull << 20)) return GUMAP_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return GUMAP_ERR_CUDA;
    auto s = std::make_unique<gumap_server>();
    s->device = device;
    s->opts.n_streams = 4;
    s->opts.max_batch_graphs = 512;
    s->opts.max_batch_vertices = 4000000;
    s->opts.max_queue = 65536;
    s->opts.staging_bytes = 512ll << 20;
    s->opts.flags = GUMAP_WEIGHTS_UNION;
    if (opts) {
        if (opts->n_streams > 0) s->opts.n_streams = opts->n_streams;
        if (opts->max_batch_graphs > 0) s->opts.max_batch_graphs = opts->max_batch_graphs;
        if (opts->max_batch_vertices > 0) s->opts.max_batch_vertices = opts->max_batch_vertices;
        if (opts->max_queue > 0) s->opts.max_queue = opts->max_queue;
        if (opts->staging_bytes > 0) s->opts.staging_bytes = opts->staging_bytes;
        s->opts.flags = opts->flags;
    }
    if (s->opts.flags & ~GUMAP_WEIGHTS_DIRECTED) return GUMAP_ERR_INVALID_ARG;
    if (cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return GUMAP_ERR_CUDA;
    const int per_sm = msbfs_max_blocks_per_sm(256);
    if (per_sm <= 0) return GUMAP_ERR_CUDA;
    s->coop_grid = s->num_sms * per_sm;
    if (batch_prepare(kBatchSmemBudget) != cudaSuccess) return GUMAP_ERR_CUDA;
    int bper = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bper, batch_kernel_ptr(), batch_threads(), kBatchSmemBudget) !=
            cudaSuccess ||
        bper < 1)
        return GUMAP_ERR_CUDA;
    s->batch_grid = s->num_sms * bper;
    if (cudaMalloc(&s->arena, hbm_budget_bytes) != cudaSuccess) return GUMAP_ERR_OOM;
    if (cudaMallocHost(&s->staging, (size_t)s->opts.staging_bytes) != cudaSuccess) {
        cudaFree(s->arena);
        return GUMAP_ERR_OOM;
    }
    s->arena_alloc.reset(hbm_budget_bytes);
    s->stage_alloc.reset((size_t)s->opts.staging_bytes);
    s->streams.resize(s->opts.n_streams);
    s->in_flight.assign(s->opts.n_streams, 0);
    for (auto& st : s->streams) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaFree(s->arena);
            cudaFreeHost(s->staging);
            return GUMAP_ERR_CUDA;
        }
    }
    s->t0 = std::chrono::steady_clock::now();
    gumap_server* raw = s.release();
    raw->worker = std::thread(scheduler, raw);
    *out = raw;
    return GUMAP_OK;
}

int gumap_serve_submit(gumap_server* s, const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                       int32_t k, int mode, uint64_t* req_id) {
    if (!s || !req_id || !row_ptr || (!col_idx && nnz > 0)) return GUMAP_ERR_INVALID_ARG;
    if (n < 2 || nnz < 0 || nnz > 0x7FFFFFFFll || k < 1 || k > GUMAP_MAX_K || k > n - 1) return GUMAP_ERR_INVALID_ARG;
    if (mode != GUMAP_FULL && mode != GUMAP_PARTIAL) return GUMAP_ERR_INVALID_ARG;
    std::string why;
    if (!host_csr_ok(row_ptr, col_idx, n, nnz, why)) return GUMAP_ERR_INVALID_GRAPH;
    auto r = std::make_unique<Request>();
    r->n = n;
    r->nnz = nnz;
    r->k = k;
    r->mode = mode;
    r->rp.assign(row_ptr, row_ptr + n + 1);
    if (nnz > 0) r->col.assign(col_idx, col_idx + nnz);
    // a request that could never be admitted, even alone
    size_t need = alone_bytes(s, r.get());
    if (is_small(r.get())) need = rows_bytes(n, k) + 8 * ((size_t)n + nnz) + (size_t)n * 4 * s->batch_grid + (1 << 20);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (need > s->arena_alloc.capacity()) return GUMAP_ERR_TOO_LARGE;
        if ((int64_t)s->waiting.size() >= s->opts.max_queue) return GUMAP_ERR_AGAIN;
        r->id = s->next_id++;
        r->t_submit = s->now();
        *req_id = r->id;
        s->waiting.push_back(r.get());
        s->reqs.emplace(r->id, std::move(r));
        s->n_submitted++;
    }
    s->cv.notify_all();
    return GUMAP_OK;
}

static int fill_result(gumap_server* s, Request* r, gumap_result* out) {
    (void)s;
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->status = r->state == 2 ? r->status : GUMAP_PENDING;
        out->n = r->n;
        out->k = r->k;
        out->t_submit = r->t_submit;
        out->t_start = r->t_start;
        out->t_done = r->t_done;
        if (r->launch) {
            out->batch_graphs = (int32_t)r->launch->reqs.size();
            out->engine = r->launch->engine;
        }
        if (r->state == 2 && r->status == GUMAP_OK && r->launch) {
            out->idx = r->launch->idx + r->row_off * r->k;
            out->dist = r->launch->dist + r->row_off * r->k;
            out->w = r->launch->w + r->row_off * r->k;
        }
    }
    return r->state == 2 ? r->status : GUMAP_PENDING;
}

int gumap_serve_poll(gumap_server* s, uint64_t req_id, gumap_result* out) {
    if (!s) return GUMAP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end() || it->second->released) return GUMAP_ERR_UNKNOWN_REQUEST;
    return fill_result(s, it->second.get(), out);
}

int gumap_serve_wait(gumap_server* s, uint64_t req_id, gumap_result* out, double timeout_s) {
    if (!s) return GUMAP_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        auto it = s->reqs.find(req_id);
        if (it == s->reqs.end() || it->second->released) return GUMAP_ERR_UNKNOWN_REQUEST;
        if (it->second->state == 2) return fill_result(s, it->second.get(), out);
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            it = s->reqs.find(req_id);
            if (it == s->reqs.end()) return GUMAP_ERR_UNKNOWN_REQUEST;
            return fill_result(s, it->second.get(), out);
        }
    }
}

int gumap_serve_read(gumap_server* s, uint64_t req_id, int32_t* idx, uint16_t* dist, float* w, void* stream) {
    if (!s) return GUMAP_ERR_INVALID_ARG;
    gumap_result r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(req_id);
        if (it == s->reqs.end() || it->second->released) return GUMAP_ERR_UNKNOWN_REQUEST;
        const int st = fill_result(s, it->second.get(), &r);
        if (st != GUMAP_OK) return st;
    }
    // the rows stay valid until the caller releases the request
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const size_t cells = (size_t)r.n * r.k;
    if (cudaSetDevice(s->device) != cudaSuccess) return GUMAP_ERR_CUDA;
    if (idx && cudaMemcpyAsync(idx, r.idx, cells * 4, cudaMemcpyDefault, cs) != cudaSuccess) return GUMAP_ERR_CUDA;
    if (dist && cudaMemcpyAsync(dist, r.dist, cells * 2, cudaMemcpyDefault, cs) != cudaSuccess) return GUMAP_ERR_CUDA;
    if (w && cudaMemcpyAsync(w, r.w, cells * 4, cudaMemcpyDefault, cs) != cudaSuccess) return GUMAP_ERR_CUDA;
    return GUMAP_OK;
}

int gumap_serve_release(gumap_server* s, uint64_t req_id) {
    if (!s) return GUMAP_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(req_id);
        if (it == s->reqs.end() || it->second->released) return GUMAP_ERR_UNKNOWN_REQUEST;
        Request* r = it->second.get();
        r->released = true;
        s->n_released++;
        if (r->state == 0) {  // never launched: drop it from the queue
            auto w = std::find(s->waiting.begin(), s->waiting.end(), r);
            if (w != s->waiting.end()) s->waiting.erase(w);
            s->reqs.erase(it);
        } else if (r->launch) {
            r->launch->n_released++;
            free_launch_if_released(s, r->launch);
        }
    }
    s->cv.notify_all();
    return GUMAP_OK;
}

double gumap_server_clock(gumap_server* s) { return s ? s->now() : 0.0; }

int gumap_server_get_stats(gumap_server* s, gumap_server_stats* out) {
    if (!s || !out) return GUMAP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->n_submitted;
    out->completed = s->n_completed;
    out->failed = s->n_failed;
    out->released = s->n_released;
    out->launches = s->n_launches;
    out->pending = (int64_t)s->waiting.size();
    int64_t running = 0;
    for (auto& L : s->launches)
        if (!L->finished) running += (int64_t)L->reqs.size();
    out->running = running;
    out->arena_bytes = (int64_t)s->arena_alloc.capacity();
    out->arena_used_bytes = (int64_t)s->arena_alloc.used();
    out->arena_peak_bytes = (int64_t)s->arena_peak;
    return GUMAP_OK;
}

int gumap_server_destroy(gumap_server* s) {
    if (!s) return GUMAP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto& L : s->launches) {  // let the scheduler drop finished launches
            L->n_released = (int)L->reqs.size();
        }
    }
    s->cv.notify_all();
    // the scheduler exits once every launch it started has completed
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (auto& L : s->launches) L->n_released = (int)L->reqs.size();
            bool all_finished = true;
            for (auto& L : s->launches)
                if (!L->finished) all_finished = false;
            if (all_finished) {
                while (!s->launches.empty()) free_launch_if_released(s, s->launches.front().get());
            }
        }
        s->cv.notify_all();
        if (s->worker.joinable()) {
            bool done;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                done = s->launches.empty();
            }
            if (done) break;
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    s->worker.join();
    cudaSetDevice(s->device);
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    cudaFree(s->arena);
    cudaFreeHost(s->staging);
    delete s;
    return GUMAP_OK;
}

}  // extern "C"
