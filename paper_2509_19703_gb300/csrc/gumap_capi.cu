// Host runtime of libgumap: the C ABI of include/gumap.h.
//
// A handle owns a device copy of the CSR graph and the scratch of the
// engines. gumap_knn_run enqueues, on the caller's stream and without any
// host synchronisation:
//   C0+C1  the BFS engine over blocks of sources (msbfs.cu, frontier.cu),
//          writing the (distance, id)-ordered kNN rows into the caller's
//          out_idx/out_dist;
//   W      rho/sigma/a_ij (weights.cu) and, for union weights, the fuzzy
//          union and the symmetric COO sorted by (row, col): an LSD radix sort
//          of (row, col) keys (sort.cu) below 2^21 slots, built row by row
//          (coo.cu) from there on.
#include "gumap.h"
#include "gumap_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace gumap;

namespace {

thread_local std::string g_last_error;

int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

}  // namespace

// Records the calling thread's last-error message for an entry point defined
// in another translation unit; returns status.
int gumap::report_error(int status, const char* msg) {
    g_last_error = msg ? msg : "";
    return status;
}

namespace {

int cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(GUMAP_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(GUMAP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
    } while (0)

int key_bits_for(int32_t n) {
    unsigned x = n > 1 ? (unsigned)(n - 1) : 1u;
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

}  // namespace

// Host-side CSR validation (same rules as the device validator).
bool gumap::host_csr_ok(const int32_t* rp, const int32_t* col, int32_t n, int64_t nnz, std::string& why) {
    if (rp[0] != 0) { why = "row_ptr[0] != 0"; return false; }
    if ((int64_t)rp[n] != nnz) { why = "row_ptr[n] != nnz"; return false; }
    for (int32_t u = 0; u < n; ++u)
        if (rp[u + 1] < rp[u]) { why = "row_ptr not monotone"; return false; }
    for (int32_t u = 0; u < n; ++u) {
        int32_t prev = -1;
        for (int32_t p = rp[u]; p < rp[u + 1]; ++p) {
            const int32_t v = col[p];
            if (v < 0 || v >= n) { why = "column id out of range"; return false; }
            if (v == u) { why = "self loop"; return false; }
            if (v <= prev) { why = "row not strictly ascending (unsorted or duplicate)"; return false; }
            prev = v;
            const int32_t* b = col + rp[v];
            const int32_t* e = col + rp[v + 1];
            const int32_t* f = std::lower_bound(b, e, u);
            if (f == e || *f != u) { why = "graph not symmetric"; return false; }
        }
    }
    return true;
}

// Units of the batched engine for graphs laid side by side: per graph, the
// widest source block whose bitsets fit a CTA's shared memory (all three,
// else frontier + next with the visited bitset in a global slab), ordered
// longest first so the work queue's tail is short. Returns -1, or the index
// of a graph too large for the engine.
int32_t gumap::plan_batch(int32_t n_graphs, const int32_t* vertex_offsets, const int64_t* graph_edges,
                          const int32_t* modes, std::vector<BatchUnit>& units_out, size_t& smem,
                          long long& slab, int32_t max_w) {
    std::vector<BatchUnit> units;
    std::vector<long long> cost;
    smem = 0;
    slab = 0;
    for (int32_t g = 0; g < n_graphs; ++g) {
        const int32_t lo = vertex_offsets[g], ng = vertex_offsets[g + 1] - lo;
        const int32_t wmax = std::min<int32_t>(std::min<int32_t>(kMaxBatchW, std::max<int32_t>(max_w, 1)), (ng + 31) / 32);
        int32_t W = 0, vg = 0;
        for (int32_t w = wmax; w >= 1 && !W; --w)
            if (4ull * (3ull * ng * w + 34ull * w) <= kBatchSmemBudget) W = w;
        if (!W) {
            vg = 1;
            for (int32_t w = wmax; w >= 1 && !W; --w)
                if (4ull * (2ull * ng * w + 34ull * w) <= kBatchSmemBudget) W = w;
        }
        if (!W) return g;
        if (W >= 4) W &= ~3;  // rows of 128-bit groups (16-byte aligned) for the batched pull
        const size_t need = 4ull * ((vg ? 2ull : 3ull) * ng * W + 34ull * W);
        smem = std::max(smem, need);
        if (vg) slab = std::max<long long>(slab, ((long long)ng * W + 3) & ~3ll);
        const long long edges = graph_edges[g];
        for (int32_t s = 0; s < ng; s += 32 * W) {
            BatchUnit u{};
            u.v0 = lo;
            u.n = ng;
            u.s_lo = s;
            u.nb = std::min<int32_t>(32 * W, ng - s);
            u.W = W;
            u.partial = modes[g] == GUMAP_PARTIAL ? 1 : 0;
            u.v_global = vg;
            units.push_back(u);
            cost.push_back((edges + ng) * W);
        }
    }
    std::vector<size_t> ord(units.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    units_out.resize(units.size());
    for (size_t i = 0; i < ord.size(); ++i) units_out[i] = units[ord[i]];
    return -1;
}

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct gumap_knn {
    int device = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t k = 1;
    int mode = GUMAP_FULL;
    uint32_t flags = 0;
    int num_sms = 0;
    int coop_grid[2][2] = {};  // resident MS-BFS CTAs: [64-bit pull items][4 CTAs per SM build]
    int opt_pull_width = 4;
    int opt_ctas_per_sm = 3;   // GUMAP_OPT_CTAS_PER_SM
    int opt_stage = 1;         // GUMAP_OPT_STAGE
    int stage_cap[2] = {};     // dynamic shared memory a staged launch may use: [4 CTAs per SM build]

    int32_t* d_rp = nullptr;
    int32_t* d_col = nullptr;
    int32_t* d_identity = nullptr;
    int32_t* d_order = nullptr;  // MS-BFS processing order (heavy vertices first)
    int32_t n_heavy = 0;
    int32_t heavy_deg = 64;
    // staged pull (see MsbfsArgs): the light vertices in processing order
    // (host copy) and, per grid size used so far, the CTA-major layout of
    // their rows: CTA b owns positions b, b + grid, b + 2 grid, ... (every
    // CTA gets the same mix of degrees), stored contiguously per CTA
    std::vector<int32_t> light_order;
    std::vector<int32_t> heavy_order;  // the hubs, whose rows the layout also holds as segments
    struct SliceCut {
        int grid;
        int32_t* d_cut;    // [grid + 1] first pair of each CTA
        int2* d_meta;      // (vertex, ocol offset) per position, CTA-major, + 3 of padding
        int32_t* d_ocol;   // the rows in that order, + 4 of padding
        size_t meta_bytes, ocol_bytes;
        int bytes;         // shared memory of the largest CTA share, rounded up to 1 KB
        int hub_segments;  // 1: the hubs' rows are in the layout as segments
    };
    std::vector<SliceCut> cuts;
    int first_grid = -1;  // a grid size launched once without its layout (built on its second launch)
    int64_t staged_launches = 0;
    std::vector<int32_t> deg;    // host copy of the vertex degrees
    DeviceCounters* d_ctr = nullptr;

    // options
    int opt_engine = GUMAP_ENGINE_AUTO;
    int64_t opt_block_bits = 0;
    int opt_profile = 0;
    // GUMAP_OPT_GRAPH: the arguments of a run, the run captured for them and
    // the host-side counts one replay stands for
    struct RunKey {
        const int32_t* src = nullptr;
        int32_t n_src = 0;
        int32_t* idx = nullptr;
        uint16_t* dist = nullptr;
        float* w = nullptr;
        cudaStream_t st = nullptr;
        bool operator==(const RunKey& o) const {
            return src == o.src && n_src == o.n_src && idx == o.idx && dist == o.dist && w == o.w && st == o.st;
        }
    };
    int opt_graph = 0;
    cudaGraphExec_t graph_exec = nullptr;
    RunKey graph_key, warm_key, refused_key;
    int warm_runs = 0;
    bool graph_refused = false;
    int64_t graph_d_kernels = 0, graph_d_bfs = 0, graph_d_staged = 0, graph_d_sort = 0;
    int64_t graph_replays = 0;
    int64_t opt_state_bytes = 0;
    // GUMAP_OPT_DIRECTION: pull only by default. Push levels are correct but
    // were slower on every measured workload: with many sources per block the
    // frontier holds most vertices even when each row holds few bits.
    int opt_direction = 1;
    int opt_push_div = 8;    // GUMAP_OPT_PUSH_DIV

    // MS-BFS scratch
    DevBuf bits;        // F, N, S
    DevBuf act, need, cnt;

    // per-run scratch
    DevBuf rho, sigma, wrow;  // wrow: the smoothing step's per-row records (union weights)
    DevBuf keys, vals, keys_tmp, vals_tmp, sort_temp;  // COO as radix-sorted (key, value) pairs
    // COO by rows (with the radix build's key and value buffers for the transposed entries)
    DevBuf coo_scr, coo_kval, coo_mcnt, coo_scol, coo_sw, coo_rowoff, coo_col, coo_w;
    // quality metrics of a drawing: per-vertex terms, all-pairs rows, kNN rows of that BFS
    DevBuf q_term, q_apsp, q_idx, q_dist;
    // spectral layout: CSR of a radix-built COO, vectors, basis, partial sums
    DevBuf sp_rowoff, sp_col, sp_vec, sp_Q, sp_part;

    // last run
    int32_t last_n_src = -1;
    bool last_union = false;
    bool coo_rows = false;  // the last run's COO was built by rows (coo), else radix-sorted pairs
    CooArgs coo{};
    unsigned long long* coo_keys = nullptr;
    float* coo_vals = nullptr;
    int coo_key_bits = 0;
    int last_engine = 0;
    int last_block_bits = 0;
    int last_blocks = 0;

    // batched engine (handles made by gumap_batch_create; a single graph's
    // handle plans itself as a one-graph batch when that engine is chosen)
    bool batch = false;
    bool batch_planned = false;
    int32_t n_graphs = 0;
    BatchUnit* d_units = nullptr;
    int32_t n_units = 0;
    size_t batch_smem = 0;
    int batch_grid = 0;
    long long vslab_words = 0;
    DevBuf vslab;
    std::vector<int32_t> batch_offsets, batch_modes;  // the batch's graphs, kept to re-plan
    std::vector<int64_t> batch_edges;
    int32_t batch_width = 0;  // GUMAP_OPT_BATCH_WIDTH in force
    int opt_coo_build = 0;    // GUMAP_OPT_COO_BUILD
    int opt_frontier_build = 0;  // GUMAP_OPT_FRONTIER_BUILD

    // Blocks replaced by a larger one while work queued before may still use
    // them: each goes back to the pool once an event recorded on the stream of
    // that work has completed (no device-wide synchronisation).
    struct Deferred {
        void* p;
        size_t bytes;
        cudaEvent_t ev;
    };
    std::vector<Deferred> deferred;
    cudaStream_t last_stream = nullptr;  // stream of the handle's latest enqueued work

    // stats
    int64_t bfs_launches = 0;
    int64_t kernel_launches = 0;
    std::vector<cudaEvent_t> ev_pool;  // pairs
    std::vector<int> ev_stage;         // per pair: what it brackets (kStage*)
    size_t ev_used = 0;
    double bfs_ms_done = 0.0;
    double weights_ms_done = 0.0;
    double sort_ms_done = 0.0;
    int64_t sort_launches = 0;
};

namespace {

// Hands the deferred blocks whose work has finished back to the pool (all of
// them when `all`: the caller has synchronised the device).
void reap(gumap_knn* h, bool all) {
    size_t keep = 0;
    for (size_t i = 0; i < h->deferred.size(); ++i) {
        const gumap_knn::Deferred d = h->deferred[i];
        if (all || cudaEventQuery(d.ev) == cudaSuccess) {
            pool_free(d.p, d.bytes);
            cudaEventDestroy(d.ev);
        } else {
            h->deferred[keep++] = d;
        }
    }
    h->deferred.resize(keep);
}

// Buffers come from the library's pool (pool.cu). A buffer that grows hands
// its old block back only once the work the handle queued before (on
// last_stream; a handle's calls are ordered on its streams by contract) has
// finished.
int ensure(gumap_knn* h, DevBuf& b, size_t bytes, const char* what) {
    if (b.bytes >= bytes && b.p) return GUMAP_OK;
    if (b.p) {
        cudaEvent_t ev = nullptr;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event for a replaced buffer");
        cudaError_t e = cudaEventRecord(ev, h->last_stream);
        if (e != cudaSuccess) {
            cudaEventDestroy(ev);
            return cuda_fail(e, "event for a replaced buffer");
        }
        h->deferred.push_back({b.p, b.bytes, ev});
        b.p = nullptr;
        b.bytes = 0;
    }
    if (bytes == 0) bytes = 16;
    CK(pool_alloc(&b.p, bytes), what);
    b.bytes = bytes;
    return GUMAP_OK;
}

// The caller guarantees the device is done with the buffer.
void release(DevBuf& b) {
    if (b.p) pool_free(b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
}

size_t held_bytes(const gumap_knn* h) {
    size_t t = (size_t)(h->n + 1) * 4 + (size_t)h->nnz * 4 + (size_t)h->n * 4 + sizeof(DeviceCounters);
    for (const auto& c : h->cuts) t += (size_t)(c.grid + 1) * 4 + c.meta_bytes + c.ocol_bytes;
    const DevBuf* bs[] = {&h->bits, &h->act, &h->need, &h->cnt, &h->rho, &h->sigma, &h->wrow,
                          &h->keys, &h->vals, &h->keys_tmp, &h->vals_tmp, &h->sort_temp,
                          &h->coo_scr, &h->coo_kval, &h->coo_mcnt, &h->coo_scol, &h->coo_sw,
                          &h->coo_rowoff, &h->coo_col, &h->coo_w, &h->q_term, &h->q_apsp, &h->q_idx, &h->q_dist,
                          &h->sp_rowoff, &h->sp_col, &h->sp_vec, &h->sp_Q, &h->sp_part};
    for (const DevBuf* b : bs) t += b->bytes;
    return t;
}

// Sources per MS-BFS block: the largest multiple of 128 whose three bitsets
// fit the state budget, balanced over the blocks the sources need. The
// default budget (256 MB) is the autotuner's choice on the 20,000-vertex
// scale-free graph: one wide block beats two L2-sized ones, because every
// block repeats the levels, the grid barriers and the extraction scans.
int choose_block_bits(const gumap_knn* h, int32_t n_src) {
    if (h->opt_block_bits > 0) return (int)h->opt_block_bits;
    const double budget = h->opt_state_bytes > 0 ? (double)h->opt_state_bytes : 256.0 * 1024 * 1024;
    long long smax = (long long)(budget * 8.0 / (3.0 * (double)std::max<int32_t>(h->n, 1)));
    smax = (smax / 128) * 128;
    if (smax < 128) smax = 128;
    if (smax > 32768) smax = 32768;
    const long long want = std::max<long long>(n_src, 1);
    const long long nblocks = (want + smax - 1) / smax;
    long long s = (want + nblocks - 1) / nblocks;
    s = ((s + 127) / 128) * 128;
    return (int)s;
}

int pick_engine(const gumap_knn* h) {
    if (h->opt_engine != GUMAP_ENGINE_AUTO) return h->opt_engine;
    if (h->batch) return GUMAP_ENGINE_BATCH;
    return h->mode == GUMAP_PARTIAL ? GUMAP_ENGINE_FRONTIER : GUMAP_ENGINE_MSBFS;
}

// What a profiling event pair brackets (GUMAP_OPT_PROFILE).
constexpr int kStageBfs = 0;      // one BFS engine launch
constexpr int kStageWeights = 1;  // rho/sigma and weights, union (with the COO row counts)
constexpr int kStageSort = 2;     // the COO build: radix sort of the pairs, or row scan, scatter, row sorts

int next_event_pair(gumap_knn* h, cudaEvent_t* a, cudaEvent_t* b, int stage = kStageBfs) {
    if (h->ev_used + 2 > h->ev_pool.size()) {
        for (int i = 0; i < 2; ++i) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e), "cudaEventCreate");
            h->ev_pool.push_back(e);
        }
        h->ev_stage.push_back(kStageBfs);
    }
    *a = h->ev_pool[h->ev_used];
    *b = h->ev_pool[h->ev_used + 1];
    h->ev_stage[h->ev_used / 2] = stage;
    h->ev_used += 2;
    return GUMAP_OK;
}

// Per-device launch limits of the MS-BFS kernel, queried once per device
// (the attribute and occupancy queries cost more than the rest of creating
// a small handle). The caller has made `device` current.
struct LaunchLimits {
    int sms = 0;
    int per_sm[2][2] = {};  // resident CTAs per SM: [64-bit pull items][4 CTAs per SM build]
    int stage_cap[2] = {};  // dynamic shared memory per CTA that keeps that residency: [4 CTAs per SM build]
};

int launch_limits(int device, LaunchLimits& out) {
    static std::mutex mu;
    static std::vector<LaunchLimits> cache;
    std::lock_guard<std::mutex> lock(mu);
    if ((size_t)device < cache.size() && cache[(size_t)device].sms > 0) {
        out = cache[(size_t)device];
        return GUMAP_OK;
    }
    LaunchLimits l;
    CK(cudaDeviceGetAttribute(&l.sms, cudaDevAttrMultiProcessorCount, device), "device attribute");
    for (int w = 0; w < 2; ++w)
        for (int c = 0; c < 2; ++c) {
            l.per_sm[w][c] = msbfs_max_blocks_per_sm(256, w ? 2 : 4, c ? 4 : 3);
            if (l.per_sm[w][c] <= 0) return fail(GUMAP_ERR_CUDA, "msbfs kernel cannot be resident");
        }
    if (l.sms <= 0) return fail(GUMAP_ERR_CUDA, "no SMs");
    // the shared memory of an SM split over the resident CTAs, less the
    // per-CTA reservation and the kernel's static arrays, in whole KB; then
    // checked (and lowered if needed) against the occupancy calculator
    int smem_sm = 0, reserved = 0, smem_block_optin = 0;
    CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device), "device attribute");
    CK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device), "device attribute");
    CK(cudaDeviceGetAttribute(&smem_block_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device), "device attribute");
    const int want3 = std::min(smem_block_optin, ((smem_sm / 3 - reserved - 512) / 1024) * 1024);
    CK(msbfs_allow_smem(want3), "kernel shared memory attribute");
    for (int c = 0; c < 2; ++c) {
        const int ctas = c ? 4 : 3;
        int cap = std::min(want3, ((smem_sm / ctas - reserved - 512) / 1024) * 1024);
        while (cap >= 16384 && (msbfs_max_blocks_per_sm(256, 4, ctas, (size_t)cap, true) < l.per_sm[0][c] ||
                                msbfs_max_blocks_per_sm(256, 2, ctas, (size_t)cap, true) < l.per_sm[1][c]))
            cap -= 4096;
        l.stage_cap[c] = cap >= 16384 ? cap : 0;
    }
    if (cache.size() <= (size_t)device) cache.resize((size_t)device + 1);
    cache[(size_t)device] = l;
    out = l;
    return GUMAP_OK;
}

void free_cuts(gumap_knn* h) {
    for (auto& c : h->cuts) {
        pool_free(c.d_cut, (size_t)(c.grid + 1) * 4);
        pool_free(c.d_meta, c.meta_bytes);
        pool_free(c.d_ocol, c.ocol_bytes);
    }
    h->cuts.clear();
}

// Processing order of the MS-BFS pull: vertices of degree > heavy_deg
// (warp-wide items) then the rest, each by decreasing degree (a counting
// sort on the host degrees, stable in vertex id). Synchronous upload. The
// staged layouts of the previous order are dropped: the caller guarantees
// no launch still uses them.
int build_order(gumap_knn* h) {
    const int32_t n = h->n;
    int32_t maxd = 0;
    for (int32_t v = 0; v < n; ++v) maxd = std::max(maxd, h->deg[v]);
    std::vector<int32_t> start((size_t)maxd + 2, 0), order((size_t)n);
    for (int32_t v = 0; v < n; ++v) start[(size_t)(maxd - h->deg[v]) + 1]++;
    for (size_t i = 1; i < start.size(); ++i) start[i] += start[i - 1];
    for (int32_t v = 0; v < n; ++v) order[(size_t)start[(size_t)(maxd - h->deg[v])]++] = v;
    int32_t nh = 0;
    while (nh < n && h->deg[order[(size_t)nh]] > h->heavy_deg) ++nh;
    h->n_heavy = nh;
    CK(cudaMemcpy(h->d_order, order.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice), "order upload");

    h->light_order.assign(order.begin() + nh, order.end());
    h->heavy_order.assign(order.begin(), order.begin() + nh);
    free_cuts(h);
    return GUMAP_OK;
}

// The staged layout for a launch of `grid` CTAs (see the handle's
// SliceCut): CTA b's positions b, b + grid, ... stored contiguously, their
// (vertex, offset) pairs uploaded and their rows gathered on stream st.
// Built at the first launch with that grid size, then kept.
int get_cut(gumap_knn* h, int grid, cudaStream_t st, const gumap_knn::SliceCut** out) {
    for (const auto& c : h->cuts)
        if (c.grid == grid) {
            *out = &c;
            return GUMAP_OK;
        }
    // positions: the hubs' segments (heaviest hubs first), then the light
    // vertices, each as (vertex or ~(hub * kHubSegMax + segment), row length)
    std::vector<int2> pos;
    const bool segs = !h->heavy_order.empty() && h->heavy_order.size() < (size_t)(INT32_MAX / kHubSegMax);
    pos.reserve(h->light_order.size() + (segs ? h->heavy_order.size() : 0));
    if (segs)
        for (size_t hh = 0; hh < h->heavy_order.size(); ++hh) {
            const int d = h->deg[(size_t)h->heavy_order[hh]];
            const int len = hub_seg_len(d), nseg = hub_seg_count(d);
            for (int sg = 0; sg < nseg; ++sg)
                pos.push_back(make_int2(~(int)(hh * kHubSegMax + sg), std::min(len, d - sg * len)));
        }
    for (int32_t v : h->light_order) pos.push_back(make_int2(v, h->deg[(size_t)v]));
    const int64_t nl = (int64_t)pos.size();
    std::vector<int2> meta((size_t)nl + 3);
    std::vector<int32_t> cut((size_t)grid + 1);
    int64_t off = 0, i = 0;
    long long worst = 0;
    for (int b = 0; b < grid; ++b) {
        cut[(size_t)b] = (int32_t)i;
        const int64_t i0 = i, off0 = off;
        for (int64_t p = b; p < nl; p += grid) {
            meta[(size_t)i++] = make_int2(pos[(size_t)p].x, (int)off);
            off += pos[(size_t)p].y;
        }
        worst = std::max(worst, stage_slice_bytes(i0, i, off0, off));
    }
    cut[(size_t)grid] = (int32_t)i;
    for (int64_t j = nl; j < nl + 3; ++j) meta[(size_t)j] = make_int2(0, (int)off);
    gumap_knn::SliceCut c{grid, nullptr, nullptr, nullptr, sizeof(int2) * meta.size(),
                          sizeof(int32_t) * ((size_t)off + 4),
                          (int)std::min<long long>(((worst + 1023) / 1024) * 1024, 1 << 30), segs ? 1 : 0};
    cudaError_t e;
    if ((e = pool_alloc((void**)&c.d_cut, (size_t)(grid + 1) * 4)) != cudaSuccess ||
        (e = pool_alloc((void**)&c.d_meta, c.meta_bytes)) != cudaSuccess ||
        (e = pool_alloc((void**)&c.d_ocol, c.ocol_bytes)) != cudaSuccess) {
        pool_free(c.d_cut, (size_t)(grid + 1) * 4);
        pool_free(c.d_meta, c.meta_bytes);
        pool_free(c.d_ocol, c.ocol_bytes);
        return cuda_fail(e, "cudaMalloc");
    }
    // the host vectors go out of scope: the copies must have read them before
    // the layout is registered (a layout whose upload failed is never kept)
    if ((e = cudaMemcpyAsync(c.d_cut, cut.data(), (size_t)(grid + 1) * 4, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(c.d_meta, meta.data(), c.meta_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(c.d_ocol + off, 0, 4 * sizeof(int32_t), st)) != cudaSuccess ||
        (e = launch_gather_rows(h->d_rp, h->d_col, h->d_order, c.d_meta, (int32_t)nl, c.d_ocol, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        pool_free(c.d_cut, (size_t)(grid + 1) * 4);
        pool_free(c.d_meta, c.meta_bytes);
        pool_free(c.d_ocol, c.ocol_bytes);
        return cuda_fail(e, "layout upload");
    }
    h->cuts.push_back(c);  // owned by the handle from here on (freed with it)
    *out = &h->cuts.back();
    return GUMAP_OK;
}

// identity: src is the handle's 0 .. n-1 (all vertices as sources); apsp: the
// all-pairs rows [n_src][n] (preset to 0xFFFF) or NULL
int run_msbfs(gumap_knn* h, const int32_t* src, bool identity, int32_t n_src, int32_t* out_idx, uint16_t* out_dist,
              cudaStream_t st, uint16_t* apsp = nullptr, bool force_full = false) {
    const int S = choose_block_bits(h, n_src);
    if (S % 128 != 0 || S <= 0) return fail(GUMAP_ERR_INVALID_ARG, "block bits must be a positive multiple of 128");
    const int W = S / 32;
    const size_t words = (size_t)h->n * W;
    int rc;
    // bitsets F, N, S, then 4 frontier queues and the queue-entry levels (n ints each), then the
    // pull items' saturation states (n x W/2 bytes: enough for either item width), 16-byte aligned
    const size_t sat_off = (words * 3 * sizeof(uint32_t) + 5 * (size_t)h->n * sizeof(int32_t) + 15) & ~(size_t)15;
    const size_t sat_bytes = ((size_t)h->n * (size_t)(W / 2) + 15) & ~(size_t)15;
    if ((rc = ensure(h, h->bits, sat_off + sat_bytes, "bitsets"))) return rc;
    if ((rc = ensure(h, h->act, (size_t)W * 4, "act"))) return rc;
    if ((rc = ensure(h, h->need, (size_t)W * 4, "need"))) return rc;
    if ((rc = ensure(h, h->cnt, (size_t)S * 4, "cnt"))) return rc;
    uint32_t* base = static_cast<uint32_t*>(h->bits.p);
    const int nblocks = (int)(((long long)n_src + S - 1) / S);
    for (int b = 0; b < nblocks; ++b) {
        MsbfsArgs a{};
        a.row_ptr = h->d_rp;
        a.col = h->d_col;
        a.n = h->n;
        a.src = src + (size_t)b * S;
        a.identity = identity ? 1 : 0;
        a.src_lo = b * S;
        a.nb = std::min<int32_t>(S, n_src - b * S);
        a.W = W;
        a.F = base;
        a.N = base + words;
        a.S = base + 2 * words;
        a.heavy = h->d_order;
        a.n_heavy = h->n_heavy;
        a.light = h->d_order + h->n_heavy;
        a.n_light = h->n - h->n_heavy;
        a.act = static_cast<uint32_t*>(h->act.p);
        a.need = static_cast<uint32_t*>(h->need.p);
        a.cnt = static_cast<int32_t*>(h->cnt.p);
        a.out_idx = out_idx + (size_t)b * S * h->k;
        a.out_dist = out_dist + (size_t)b * S * h->k;
        a.k = h->k;
        a.partial = (h->mode == GUMAP_PARTIAL && !force_full) ? 1 : 0;
        a.apsp = apsp ? apsp + (size_t)b * S * (size_t)h->n : nullptr;
        a.apsp_ld = h->n;
        a.ctr = h->d_ctr;
        a.direction = h->opt_direction;
        a.push_div = h->opt_push_div;
        a.pull_width = h->opt_pull_width;
        a.ctas_per_sm = h->opt_ctas_per_sm;
        a.queue = reinterpret_cast<int32_t*>(base + 3 * words);
        a.inq = a.queue + 4 * (size_t)h->n;
        a.sat = reinterpret_cast<uint8_t*>(h->bits.p) + sat_off;
        // pull-only levels over consecutive sources pull from the seen sets
        a.seen_only = (identity && h->opt_direction == 1) ? 1 : 0;
        const int grid = msbfs_grid_for(a, h->coop_grid[a.pull_width == 2][a.ctas_per_sm == 4]);
        const int cap = h->stage_cap[a.ctas_per_sm == 4];
        // The layout costs host work, uploads and a stream synchronisation, so a
        // grid size's first launch reads the rows from the CSR and its second
        // launch builds the layout: a handle that runs once never pays for it.
        bool layout = false;
        for (const auto& c : h->cuts) layout = layout || c.grid == grid;
        if (!layout && h->first_grid != grid) {
            h->first_grid = grid;
        } else if (h->opt_stage && h->n > h->n_heavy && cap > 0) {
            const gumap_knn::SliceCut* c = nullptr;
            if ((rc = get_cut(h, grid, st, &c))) return rc;
            if (c->bytes <= cap) {
                a.staged = h->opt_stage;
                a.stage_bytes = c->bytes;
                a.meta = c->d_meta;
                a.ocol = c->d_ocol;
                a.slice = c->d_cut;
                a.hub_segments = c->hub_segments;
                h->staged_launches++;
            }
        }
        CK(cudaMemsetAsync(h->d_ctr, 0, kLaunchCounterBytes, st), "reset barrier");
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->opt_profile) {
            if ((rc = next_event_pair(h, &e0, &e1))) return rc;
            CK(cudaEventRecord(e0, st), "cudaEventRecord");
        }
        CK(launch_msbfs(a, grid, 256, st),
           "msbfs launch");
        if (h->opt_profile) CK(cudaEventRecord(e1, st), "cudaEventRecord");
        h->bfs_launches++;
        h->kernel_launches++;
    }
    h->last_block_bits = S;
    h->last_blocks = nblocks;
    return GUMAP_OK;
}

int run_batch(gumap_knn* h, int32_t* out_idx, uint16_t* out_dist, cudaStream_t st) {
    BatchArgs a{};
    a.row_ptr = h->d_rp;
    a.col = h->d_col;
    a.units = h->d_units;
    a.n_units = h->n_units;
    a.k = h->k;
    a.out_idx = out_idx;
    a.out_dist = out_dist;
    a.vslab = static_cast<uint32_t*>(h->vslab.p);
    a.vslab_words = h->vslab_words;
    a.next_unit = &h->d_ctr->aux_count;
    a.ctr = h->d_ctr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc;
    if (h->opt_profile) {
        if ((rc = next_event_pair(h, &e0, &e1))) return rc;
        CK(cudaEventRecord(e0, st), "cudaEventRecord");
    }
    CK(launch_batch(a, h->batch_grid, h->batch_smem, st), "batch launch");
    if (h->opt_profile) CK(cudaEventRecord(e1, st), "cudaEventRecord");
    h->bfs_launches++;
    h->kernel_launches++;
    h->last_block_bits = 0;
    h->last_blocks = h->n_units;
    return GUMAP_OK;
}

int run_frontier(gumap_knn* h, const int32_t* src, int32_t n_src, int32_t* out_idx, uint16_t* out_dist,
                 cudaStream_t st) {
    FrontierArgs a{};
    a.row_ptr = h->d_rp;
    a.col = h->d_col;
    a.n = h->n;
    a.src = src;
    a.n_src = n_src;
    a.k = h->k;
    a.out_idx = out_idx;
    a.out_dist = out_dist;
    a.status = &h->d_ctr->status;
    a.build = h->opt_frontier_build;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc;
    if (h->opt_profile) {
        if ((rc = next_event_pair(h, &e0, &e1))) return rc;
        CK(cudaEventRecord(e0, st), "cudaEventRecord");
    }
    CK(launch_frontier(a, st), "frontier launch");
    if (h->opt_profile) CK(cudaEventRecord(e1, st), "cudaEventRecord");
    h->bfs_launches++;
    h->kernel_launches++;
    h->last_block_bits = 0;
    h->last_blocks = 1;
    return GUMAP_OK;
}

}  // namespace

namespace {

int run_path(gumap_knn* h, const int32_t* sources, int32_t n_src, int32_t* out_idx, uint16_t* out_dist, float* out_w,
             cudaStream_t st) {
    const bool want_union = !(h->flags & GUMAP_WEIGHTS_DIRECTED);
    const int32_t* src = sources ? sources : h->d_identity;
    const int32_t k = h->k;
    int rc;
    const size_t slots = (size_t)n_src * k;
    if ((rc = ensure(h, h->rho, (size_t)n_src * 4, "rho")) || (rc = ensure(h, h->sigma, (size_t)n_src * 4, "sigma")))
        return rc;
    if (want_union && (rc = ensure(h, h->wrow, (size_t)n_src * sizeof(WeightRow), "row records"))) return rc;

    const int engine = pick_engine(h);
    h->last_engine = engine;
    if (engine == GUMAP_ENGINE_MSBFS) {
        rc = run_msbfs(h, src, sources == nullptr, n_src, out_idx, out_dist, st);
    } else if (engine == GUMAP_ENGINE_FRONTIER) {
        if (h->mode != GUMAP_PARTIAL) return fail(GUMAP_ERR_INVALID_ARG, "the frontier engine computes the partial form only");
        rc = run_frontier(h, src, n_src, out_idx, out_dist, st);
    } else if (engine == GUMAP_ENGINE_BATCH) {
        if (sources) {
            // the batched engine runs every vertex of its units; a single graph's
            // explicit sources go to the MS-BFS engine
            if (h->batch) return fail(GUMAP_ERR_INVALID_ARG, "the batched engine needs sources == NULL");
            h->last_engine = GUMAP_ENGINE_MSBFS;
            rc = run_msbfs(h, src, false, n_src, out_idx, out_dist, st);
        } else {
            rc = run_batch(h, out_idx, out_dist, st);
        }
    } else {
        return fail(GUMAP_ERR_INVALID_ARG, "engine %d not available", engine);
    }
    if (rc) return rc;

    const float T = (float)std::log2((double)k);
    WeightRow* wrow = want_union ? static_cast<WeightRow*>(h->wrow.p) : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->opt_profile) {
        if ((rc = next_event_pair(h, &e0, &e1, kStageWeights))) return rc;
        CK(cudaEventRecord(e0, st), "cudaEventRecord");
    }
    CK(launch_smooth_knn(out_idx, out_dist, n_src, k, T, static_cast<float*>(h->rho.p), static_cast<float*>(h->sigma.p),
                         wrow, want_union ? nullptr : out_w, st),
       "smooth_knn");
    h->kernel_launches++;
    const bool coo_by_rows =
        h->opt_coo_build == 2 || (h->opt_coo_build == 0 && (long long)slots >= kCooRowsMinSlots);
    if (want_union && !coo_by_rows) {
        const long long cnt = 2ll * n_src * k;
        const int B = key_bits_for(h->n);
        if ((rc = ensure(h, h->keys, cnt * 8, "coo keys")) || (rc = ensure(h, h->vals, cnt * 4, "coo vals")) ||
            (rc = ensure(h, h->keys_tmp, cnt * 8, "coo keys tmp")) || (rc = ensure(h, h->vals_tmp, cnt * 4, "coo vals tmp")) ||
            (rc = ensure(h, h->sort_temp, radix_sort_temp_bytes(cnt, 2 * B), "sort temp")))
            return rc;
        CK(cudaMemsetAsync(&h->d_ctr->coo_nnz, 0, sizeof(unsigned long long), st), "memset nnz");
        CK(launch_union_pairs(out_idx, out_dist, wrow, n_src, k, out_w, B,
                              static_cast<unsigned long long*>(h->keys.p), static_cast<float*>(h->vals.p), h->d_ctr,
                              st),
           "union");
        h->kernel_launches++;
        if (h->opt_profile) {
            CK(cudaEventRecord(e1, st), "cudaEventRecord");
            if ((rc = next_event_pair(h, &e0, &e1, kStageSort))) return rc;
            CK(cudaEventRecord(e0, st), "cudaEventRecord");
        }
        int launches = 0;
        CK(radix_sort_pairs(static_cast<unsigned long long*>(h->keys.p), static_cast<float*>(h->vals.p),
                            static_cast<unsigned long long*>(h->keys_tmp.p), static_cast<float*>(h->vals_tmp.p), cnt,
                            2 * B, h->sort_temp.p, h->sort_temp.bytes, &h->d_ctr->status, st, &h->coo_keys,
                            &h->coo_vals, &launches),
           "radix sort");
        h->kernel_launches += launches;
        h->sort_launches += launches;
        h->coo_key_bits = B;
        h->coo_rows = false;
        h->last_union = true;
    } else if (want_union) {
        const size_t slots2 = 2 * slots;
        const int TB = key_bits_for(n_src + 1);  // target bits of a mirror key: 2^TB > n
        // one zeroed block: the COO build's row ranges and scan words, then the
        // union's look-back words, its tile counter and the mirror total
        const size_t coo_bytes = coo_scratch_bytes(n_src);
        const size_t uscan_words = union_scan_words(n_src, k);
        const size_t scr_bytes = coo_bytes + (uscan_words + 2) * sizeof(unsigned long long);
        if ((rc = ensure(h, h->coo_scr, scr_bytes, "coo scratch")) ||
            (rc = ensure(h, h->coo_kval, (size_t)n_src * 4, "coo kval")) ||
            (rc = ensure(h, h->coo_mcnt, (size_t)n_src * 4, "coo mirror counts")) ||
            (rc = ensure(h, h->keys, slots * 8, "coo mirror keys")) ||
            (rc = ensure(h, h->vals, slots * 4, "coo mirror weights")) ||
            (rc = ensure(h, h->keys_tmp, slots * 8, "coo keys tmp")) ||
            (rc = ensure(h, h->vals_tmp, slots * 4, "coo vals tmp")) ||
            (rc = ensure(h, h->sort_temp, radix_sort_temp_bytes((long long)slots, TB), "sort temp")) ||
            (rc = ensure(h, h->coo_scol, slots * 4, "coo own columns")) ||
            (rc = ensure(h, h->coo_sw, slots * 4, "coo own weights")) ||
            (rc = ensure(h, h->coo_rowoff, ((size_t)n_src + 1) * 8, "coo rowoff")) ||
            (rc = ensure(h, h->coo_col, slots2 * 4, "coo cols")) || (rc = ensure(h, h->coo_w, slots2 * 4, "coo weights")))
            return rc;
        LaunchLimits lim;
        if ((rc = launch_limits(h->device, lim))) return rc;
        unsigned long long* uwords =
            reinterpret_cast<unsigned long long*>(static_cast<char*>(h->coo_scr.p) + coo_bytes);
        UnionScan us{};
        us.pub = uwords;
        us.tile_ctr = reinterpret_cast<unsigned int*>(uwords + uscan_words);
        us.total = uwords + uscan_words + 1;
        us.status = &h->d_ctr->status;
        us.limit_ns = 1000ull * 1000ull * 1000ull;
        CooArgs c{};
        coo_scratch_split(h->coo_scr.p, n_src, &c.instart, &c.inend, &c.ctr, &c.pub);
        c.idx = out_idx;
        c.w = out_w;
        c.kval = static_cast<int32_t*>(h->coo_kval.p);
        c.n = n_src;
        c.k = k;
        c.key_bits = TB;
        c.mirrors = us.total;
        c.mcnt = static_cast<uint32_t*>(h->coo_mcnt.p);
        c.scol = static_cast<int32_t*>(h->coo_scol.p);
        c.sw = static_cast<float*>(h->coo_sw.p);
        c.rowoff = static_cast<unsigned long long*>(h->coo_rowoff.p);
        c.ccol = static_cast<int32_t*>(h->coo_col.p);
        c.cw = static_cast<float*>(h->coo_w.p);
        c.status = &h->d_ctr->status;
        CK(cudaMemsetAsync(h->coo_scr.p, 0, scr_bytes, st), "memset coo scratch");
        CK(launch_union_mirrors(out_idx, out_dist, wrow, n_src, k, out_w, static_cast<int32_t*>(h->coo_kval.p),
                                static_cast<unsigned long long*>(h->keys.p), static_cast<float*>(h->vals.p), us, st),
           "union");
        h->kernel_launches++;
        if (h->opt_profile) {
            CK(cudaEventRecord(e1, st), "cudaEventRecord");
            if ((rc = next_event_pair(h, &e0, &e1, kStageSort))) return rc;
            CK(cudaEventRecord(e0, st), "cudaEventRecord");
        }
        int launches = 0;
        unsigned long long* tkey = nullptr;
        float* tval = nullptr;
        CK(radix_sort_pairs(static_cast<unsigned long long*>(h->keys.p), static_cast<float*>(h->vals.p),
                            static_cast<unsigned long long*>(h->keys_tmp.p), static_cast<float*>(h->vals_tmp.p),
                            (long long)slots, TB, h->sort_temp.p, h->sort_temp.bytes, &h->d_ctr->status, st, &tkey,
                            &tval, &launches, us.total),
           "mirror sort");
        c.tkey = tkey;
        c.tval = tval;
        CK(launch_coo_build(c, lim.sms, st, &launches), "coo build");
        h->kernel_launches += launches;
        h->sort_launches += launches;
        h->coo = c;
        h->coo_rows = true;
        h->last_union = true;
    }
    if (h->opt_profile) CK(cudaEventRecord(e1, st), "cudaEventRecord");
    return GUMAP_OK;
}

// GUMAP_OPT_GRAPH: forget the captured run (any call that may change the
// handle's buffers or the state a replay relies on does this first).
void drop_graph(gumap_knn* h) {
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
}

// Any other call on the handle: the captured run and the warm-up count go.
void forget_runs(gumap_knn* h) {
    drop_graph(h);
    h->warm_runs = 0;
}

// Capture one run of `key` into a CUDA graph and launch it. The run's
// buffers exist (two runs with the same arguments came before), so
// run_path issues only stream-ordered work. Returns false, with no work
// issued and the host counters as they were, when the capture or the
// instantiation is refused; the caller then runs normally.
bool capture_run(gumap_knn* h, const gumap_knn::RunKey& key) {
    const int64_t k0 = h->kernel_launches, b0 = h->bfs_launches, s0 = h->staged_launches, o0 = h->sort_launches;
    if (cudaStreamBeginCapture(key.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int rc = run_path(h, key.src, key.n_src, key.idx, key.dist, key.w, key.st);
    cudaGraph_t g = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(key.st, &g);
    cudaGraphExec_t ex = nullptr;
    const bool ok = rc == GUMAP_OK && e_end == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    const int64_t dk = h->kernel_launches - k0, db = h->bfs_launches - b0, ds = h->staged_launches - s0,
                  dso = h->sort_launches - o0;
    h->kernel_launches = k0;
    h->bfs_launches = b0;
    h->staged_launches = s0;
    h->sort_launches = o0;
    if (!ok || cudaGraphLaunch(ex, key.st) != cudaSuccess) {
        if (ex) cudaGraphExecDestroy(ex);
        cudaGetLastError();
        return false;
    }
    h->graph_exec = ex;
    h->graph_key = key;
    h->graph_d_kernels = dk;
    h->graph_d_bfs = db;
    h->graph_d_staged = ds;
    h->graph_d_sort = dso;
    h->kernel_launches += dk;
    h->bfs_launches += db;
    h->staged_launches += ds;
    h->sort_launches += dso;
    return true;
}

}  // namespace

extern "C" {

const char* gumap_status_string(int s) {
    switch (s) {
        case GUMAP_OK: return "GUMAP_OK";
        case GUMAP_ERR_INVALID_ARG: return "GUMAP_ERR_INVALID_ARG";
        case GUMAP_ERR_INVALID_GRAPH: return "GUMAP_ERR_INVALID_GRAPH";
        case GUMAP_ERR_OOM: return "GUMAP_ERR_OOM";
        case GUMAP_ERR_CUDA: return "GUMAP_ERR_CUDA";
        case GUMAP_ERR_AGAIN: return "GUMAP_ERR_AGAIN";
        case GUMAP_PENDING: return "GUMAP_PENDING";
        case GUMAP_ERR_TIMEOUT: return "GUMAP_ERR_TIMEOUT";
        case GUMAP_ERR_TOO_LARGE: return "GUMAP_ERR_TOO_LARGE";
        case GUMAP_ERR_UNKNOWN_REQUEST: return "GUMAP_ERR_UNKNOWN_REQUEST";
        default: return "GUMAP_ERR_UNKNOWN_STATUS";
    }
}

const char* gumap_last_error(void) { return g_last_error.c_str(); }

int gumap_knn_destroy(gumap_knn* h) {
    if (!h) return GUMAP_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();  // nothing queued may still use the buffers handed back below
    drop_graph(h);
    reap(h, true);
    pool_free(h->d_rp, sizeof(int32_t) * ((size_t)h->n + 2));
    pool_free(h->d_col, sizeof(int32_t) * (size_t)std::max<int64_t>(h->nnz, 1));
    pool_free(h->d_identity, sizeof(int32_t) * (size_t)h->n);
    pool_free(h->d_order, sizeof(int32_t) * (size_t)h->n);
    free_cuts(h);
    pool_free(h->d_units, sizeof(BatchUnit) * (size_t)std::max<int32_t>(h->n_units, 1));
    release(h->vslab);
    pool_free(h->d_ctr, sizeof(DeviceCounters));
    DevBuf* bs[] = {&h->bits, &h->act, &h->need, &h->cnt, &h->rho, &h->sigma, &h->wrow,
                    &h->keys, &h->vals, &h->keys_tmp, &h->vals_tmp, &h->sort_temp,
                    &h->coo_scr, &h->coo_kval, &h->coo_mcnt, &h->coo_scol, &h->coo_sw,
                    &h->coo_rowoff, &h->coo_col, &h->coo_w, &h->q_term, &h->q_apsp, &h->q_idx, &h->q_dist,
                    &h->sp_rowoff, &h->sp_col, &h->sp_vec, &h->sp_Q, &h->sp_part};
    for (DevBuf* b : bs) release(*b);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    delete h;
    return GUMAP_OK;
}

int gumap_knn_create(gumap_knn** out, const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                     int32_t k, int mode, uint32_t flags, int device) {
    if (!out) return fail(GUMAP_ERR_INVALID_ARG, "h is NULL");
    *out = nullptr;
    if (!row_ptr || (!col_idx && nnz > 0)) return fail(GUMAP_ERR_INVALID_ARG, "NULL CSR pointer");
    if (n < 2) return fail(GUMAP_ERR_INVALID_ARG, "n must be >= 2 (got %d)", n);
    if (nnz < 0 || nnz > 0x7FFFFFFFll) return fail(GUMAP_ERR_INVALID_ARG, "nnz out of range");
    if (k < 1 || k > GUMAP_MAX_K || k > n - 1) return fail(GUMAP_ERR_INVALID_ARG, "k must be in [1, min(n-1, %d)]", GUMAP_MAX_K);
    if (mode != GUMAP_FULL && mode != GUMAP_PARTIAL) return fail(GUMAP_ERR_INVALID_ARG, "bad mode");
    if (flags & ~(GUMAP_WEIGHTS_DIRECTED | GUMAP_CSR_ON_DEVICE | GUMAP_EMIT_APSP))
        return fail(GUMAP_ERR_INVALID_ARG, "unknown flag");
    if ((flags & GUMAP_EMIT_APSP) && mode != GUMAP_FULL)
        return fail(GUMAP_ERR_INVALID_ARG, "all-pairs rows need the full form");
    if (2ll * n * k > 0x7FFFFFFFll * 2) return fail(GUMAP_ERR_INVALID_ARG, "n * k too large");
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(GUMAP_ERR_INVALID_ARG, "bad device %d", device);
    CK(cudaSetDevice(device), "cudaSetDevice");

    if (!(flags & GUMAP_CSR_ON_DEVICE)) {
        std::string why;
        if (!host_csr_ok(row_ptr, col_idx, n, nnz, why)) return fail(GUMAP_ERR_INVALID_GRAPH, "invalid CSR: %s", why.c_str());
    }
    gumap_knn* h = new (std::nothrow) gumap_knn();
    if (!h) return fail(GUMAP_ERR_OOM, "host allocation");
    h->device = device;
    h->n = n;
    h->nnz = nnz;
    h->k = k;
    h->mode = mode;
    h->flags = flags;
    LaunchLimits lim;
    if (int lrc = launch_limits(device, lim)) {
        gumap_knn_destroy(h);
        return lrc;
    }
    h->num_sms = lim.sms;
    for (int w = 0; w < 2; ++w)
        for (int c = 0; c < 2; ++c) h->coop_grid[w][c] = lim.sms * lim.per_sm[w][c];
    h->stage_cap[0] = lim.stage_cap[0];
    h->stage_cap[1] = lim.stage_cap[1];
    cudaError_t e;

    const cudaMemcpyKind kind = (flags & GUMAP_CSR_ON_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // row_ptr plus one slot for the device validation's result
    if ((e = pool_alloc((void**)&h->d_rp, sizeof(int32_t) * ((size_t)n + 2))) != cudaSuccess ||
        (e = pool_alloc((void**)&h->d_col, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1))) != cudaSuccess ||
        (e = pool_alloc((void**)&h->d_identity, sizeof(int32_t) * (size_t)n)) != cudaSuccess ||
        (e = pool_alloc((void**)&h->d_ctr, sizeof(DeviceCounters))) != cudaSuccess) {
        gumap_knn_destroy(h);
        return cuda_fail(e, "cudaMalloc");
    }
    if ((e = cudaMemcpy(h->d_rp, row_ptr, sizeof(int32_t) * (n + 1), kind)) != cudaSuccess ||
        (nnz > 0 && (e = cudaMemcpy(h->d_col, col_idx, sizeof(int32_t) * nnz, kind)) != cudaSuccess) ||
        (e = cudaMemset(h->d_ctr, 0, sizeof(DeviceCounters))) != cudaSuccess ||
        (e = launch_identity(h->d_identity, n, 0)) != cudaSuccess) {
        gumap_knn_destroy(h);
        return cuda_fail(e, "upload");
    }
    if ((e = pool_alloc((void**)&h->d_order, sizeof(int32_t) * (size_t)n)) != cudaSuccess) {
        gumap_knn_destroy(h);
        return cuda_fail(e, "cudaMalloc");
    }
    {
        // A CSR on the device is validated there; the result lands in the slot
        // after row_ptr, so one readback brings back both (the host needs
        // row_ptr for the degrees).
        std::vector<int32_t> rp_dev;
        const int32_t* rp = row_ptr;
        if (flags & GUMAP_CSR_ON_DEVICE) {
            rp_dev.resize((size_t)n + 2);
            if ((e = launch_validate_csr(h->d_rp, h->d_col, n, nnz, h->d_rp + n + 1, 0)) != cudaSuccess ||
                (e = cudaMemcpy(rp_dev.data(), h->d_rp, sizeof(int32_t) * ((size_t)n + 2), cudaMemcpyDeviceToHost)) !=
                    cudaSuccess) {
                gumap_knn_destroy(h);
                return cuda_fail(e, "device CSR validation");
            }
            if (rp_dev[(size_t)n + 1]) {
                gumap_knn_destroy(h);
                return fail(GUMAP_ERR_INVALID_GRAPH, "invalid CSR (device validation)");
            }
            rp = rp_dev.data();
        }
        h->deg.resize((size_t)n);
        for (int32_t v = 0; v < n; ++v) h->deg[(size_t)v] = rp[(size_t)v + 1] - rp[(size_t)v];
    }
    // A vertex is "heavy" (one warp per item) only when its degree is well
    // above the graph's mean: on a uniform dense graph every vertex is long
    // but the thread-per-item pull keeps more loads in flight.
    h->heavy_deg = (int32_t)std::max<int64_t>(64, 4 * (nnz / std::max<int32_t>(n, 1)));
    int rc = build_order(h);
    if (rc) {
        gumap_knn_destroy(h);
        return rc;
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        gumap_knn_destroy(h);
        return cuda_fail(e, "create");
    }
    tune_apply_cached(h, std::getenv("GUMAP_TUNE_CACHE"));  // settings of a tuned graph of this shape
    *out = h;
    return GUMAP_OK;
}

// Cuts a batch handle's graphs into units of at most max_w words (32 max_w
// sources) and sets up the launch: shared memory, grid, visited slab, unit
// table. The device must be done with the previous plan's buffers.
int apply_batch_plan(gumap_knn* h, int32_t max_w) {
    std::vector<BatchUnit> sorted;
    size_t smem = 0;
    long long slab = 0;
    const int32_t ng = (int32_t)h->batch_modes.size();
    const int32_t big =
        plan_batch(ng, h->batch_offsets.data(), h->batch_edges.data(), h->batch_modes.data(), sorted, smem, slab, max_w);
    if (big >= 0)
        return fail(GUMAP_ERR_TOO_LARGE, "graph %d (%d vertices) does not fit the batched engine", big,
                    h->batch_offsets[(size_t)big + 1] - h->batch_offsets[(size_t)big]);
    cudaError_t e;
    CK(batch_prepare(smem), "batch kernel attributes");
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_ptr(), batch_threads(), smem),
       "batch occupancy");
    if (per_sm < 1) return fail(GUMAP_ERR_CUDA, "batch kernel cannot be resident");
    h->batch_grid = h->num_sms * per_sm;
    h->batch_smem = smem;
    h->vslab_words = slab;
    int rc;
    if (slab > 0 && (rc = ensure(h, h->vslab, (size_t)slab * 4 * h->batch_grid, "batch slab"))) return rc;
    pool_free(h->d_units, sizeof(BatchUnit) * (size_t)std::max<int32_t>(h->n_units, 1));
    h->d_units = nullptr;
    h->n_units = (int32_t)sorted.size();  // sizes the block handed back by destroy
    if ((e = pool_alloc((void**)&h->d_units, sizeof(BatchUnit) * sorted.size())) != cudaSuccess) {
        h->n_units = 0;
        return cuda_fail(e, "batch units");
    }
    CK(cudaMemcpy(h->d_units, sorted.data(), sizeof(BatchUnit) * sorted.size(), cudaMemcpyHostToDevice),
       "batch units");
    h->batch_width = max_w;
    h->batch_planned = true;
    return GUMAP_OK;
}

int gumap_batch_create(gumap_knn** out, int32_t n_graphs, const int32_t* vertex_offsets, const int32_t* row_ptr,
                       const int32_t* col_idx, int64_t nnz, int32_t k, const int32_t* modes, uint32_t flags,
                       int device) {
    if (!out) return fail(GUMAP_ERR_INVALID_ARG, "h is NULL");
    *out = nullptr;
    if (n_graphs < 1 || !vertex_offsets || !modes) return fail(GUMAP_ERR_INVALID_ARG, "bad graph list");
    if (flags & GUMAP_CSR_ON_DEVICE) return fail(GUMAP_ERR_INVALID_ARG, "batch CSR must be on the host");
    if (vertex_offsets[0] != 0) return fail(GUMAP_ERR_INVALID_ARG, "vertex_offsets[0] != 0");
    for (int32_t g = 0; g < n_graphs; ++g) {
        if (vertex_offsets[g + 1] <= vertex_offsets[g]) return fail(GUMAP_ERR_INVALID_ARG, "graph %d is empty", g);
        if (modes[g] != GUMAP_FULL && modes[g] != GUMAP_PARTIAL) return fail(GUMAP_ERR_INVALID_ARG, "bad mode of graph %d", g);
    }
    const int32_t n = vertex_offsets[n_graphs];
    gumap_knn* h = nullptr;
    int rc = gumap_knn_create(&h, row_ptr, col_idx, n, nnz, k, GUMAP_FULL, flags, device);
    if (rc) return rc;
    // no edge may leave its graph (rows are sorted: checking each row's ends suffices)
    for (int32_t g = 0; g < n_graphs; ++g) {
        const int32_t lo = vertex_offsets[g], hi = vertex_offsets[g + 1];
        for (int32_t v = lo; v < hi; ++v) {
            if (row_ptr[v + 1] > row_ptr[v] && (col_idx[row_ptr[v]] < lo || col_idx[row_ptr[v + 1] - 1] >= hi)) {
                gumap_knn_destroy(h);
                return fail(GUMAP_ERR_INVALID_GRAPH, "an edge of vertex %d leaves its graph %d", v, g);
            }
        }
    }
    h->batch_offsets.assign(vertex_offsets, vertex_offsets + n_graphs + 1);
    h->batch_modes.assign(modes, modes + n_graphs);
    h->batch_edges.resize((size_t)n_graphs);
    for (int32_t g = 0; g < n_graphs; ++g)
        h->batch_edges[(size_t)g] = (int64_t)row_ptr[vertex_offsets[g + 1]] - row_ptr[vertex_offsets[g]];
    if ((rc = apply_batch_plan(h, kMaxBatchW))) {
        gumap_knn_destroy(h);
        return rc;
    }
    h->batch = true;
    h->n_graphs = n_graphs;
    *out = h;
    return GUMAP_OK;
}

int gumap_knn_run(gumap_knn* h, const int32_t* sources, int32_t n_src, int32_t* out_idx, uint16_t* out_dist,
                  float* out_w, void* stream) {
    if (!h) return fail(GUMAP_ERR_INVALID_ARG, "NULL handle");
    if (n_src < 0) return fail(GUMAP_ERR_INVALID_ARG, "n_src < 0");
    if (n_src == 0) {  // nothing to compute; pointers may be NULL
        h->last_n_src = 0;
        h->last_union = false;
        return GUMAP_OK;
    }
    if (!sources && n_src != h->n) return fail(GUMAP_ERR_INVALID_ARG, "sources == NULL requires n_src == n");
    const bool want_union = !(h->flags & GUMAP_WEIGHTS_DIRECTED);
    if (want_union && sources) return fail(GUMAP_ERR_INVALID_ARG, "union weights need sources == NULL (all vertices)");
    if (n_src > 0 && (!out_idx || !out_dist || !out_w)) return fail(GUMAP_ERR_INVALID_ARG, "NULL output");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    reap(h, false);
    gumap_knn::RunKey key;
    key.src = sources;
    key.n_src = n_src;
    key.idx = out_idx;
    key.dist = out_dist;
    key.w = out_w;
    key.st = st;
    const bool graphs = h->opt_graph && !h->opt_profile && st != nullptr;
    if (graphs && h->graph_exec && h->graph_key == key) {  // replay the captured run
        CK(cudaGraphLaunch(h->graph_exec, st), "cudaGraphLaunch");
        h->kernel_launches += h->graph_d_kernels;
        h->bfs_launches += h->graph_d_bfs;
        h->staged_launches += h->graph_d_staged;
        h->sort_launches += h->graph_d_sort;
        h->graph_replays++;
        h->last_stream = st;
        return GUMAP_OK;
    }
    drop_graph(h);
    h->last_n_src = n_src;
    h->last_union = false;
    if (graphs && h->warm_key == key && h->warm_runs >= 2 && !(h->graph_refused && h->refused_key == key)) {
        if (capture_run(h, key)) {
            h->graph_replays++;
            h->last_stream = st;
            return GUMAP_OK;
        }
        h->graph_refused = true;  // this run's capture was refused: run it, and it, normally from now on
        h->refused_key = key;
        h->last_n_src = n_src;
        h->last_union = false;
    }
    const int rc = run_path(h, sources, n_src, out_idx, out_dist, out_w, st);
    h->last_stream = st;
    if (graphs && rc == GUMAP_OK) {
        h->warm_runs = h->warm_key == key ? h->warm_runs : 0;
        h->warm_key = key;
        h->warm_runs++;
    }
    return rc;
}

int gumap_knn_apsp(gumap_knn* h, const int32_t* sources, int32_t n_src, int32_t* out_idx, uint16_t* out_dist,
                   uint16_t* out_apsp, void* stream) {
    if (!h) return fail(GUMAP_ERR_INVALID_ARG, "NULL handle");
    forget_runs(h);  // a captured run may not outlive this call (GUMAP_OPT_GRAPH)
    if (!(h->flags & GUMAP_EMIT_APSP)) return fail(GUMAP_ERR_INVALID_ARG, "handle not created with GUMAP_EMIT_APSP");
    if (h->batch) return fail(GUMAP_ERR_INVALID_ARG, "all-pairs rows of a batch handle are not available");
    if (h->n > 65535) return fail(GUMAP_ERR_INVALID_ARG, "all-pairs rows need n <= 65535 (uint16 distances)");
    if (n_src < 0) return fail(GUMAP_ERR_INVALID_ARG, "n_src < 0");
    if (n_src == 0) return GUMAP_OK;
    if (!sources && n_src != h->n) return fail(GUMAP_ERR_INVALID_ARG, "sources == NULL requires n_src == n");
    if (!out_idx || !out_dist || !out_apsp) return fail(GUMAP_ERR_INVALID_ARG, "NULL output");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaMemsetAsync(out_apsp, 0xFF, (size_t)n_src * (size_t)h->n * sizeof(uint16_t), st), "preset rows");
    h->last_n_src = -1;  // no weights: rho_sigma and coo refer to no run
    h->last_union = false;
    h->last_engine = GUMAP_ENGINE_MSBFS;
    reap(h, false);
    const int rc = run_msbfs(h, sources ? sources : h->d_identity, sources == nullptr, n_src, out_idx, out_dist, st,
                             out_apsp);
    h->last_stream = st;
    return rc;
}

int gumap_quality_np(gumap_knn* h, const float* X, int32_t dim, int32_t r, int32_t* out_c, int32_t* out_inter,
                     double* out_sum, void* stream) {
    if (!h) return fail(GUMAP_ERR_INVALID_ARG, "NULL handle");
    forget_runs(h);  // a captured run may not outlive this call (GUMAP_OPT_GRAPH)
    if (h->batch) return fail(GUMAP_ERR_INVALID_ARG, "quality metrics take a single graph's handle");
    if (!X || !out_sum) return fail(GUMAP_ERR_INVALID_ARG, "NULL drawing or output");
    if (dim < 1 || dim > 8) return fail(GUMAP_ERR_INVALID_ARG, "dim must be in [1, 8]");
    if (r < 1) return fail(GUMAP_ERR_INVALID_ARG, "r must be >= 1");
    if (h->n > (1 << 20)) return fail(GUMAP_ERR_INVALID_ARG, "neighbourhood preservation takes n <= 2^20");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    reap(h, false);
    int rc;
    if ((rc = ensure(h, h->q_term, (size_t)h->n * sizeof(double), "np terms"))) return rc;
    CK(launch_np(h->d_rp, h->d_col, h->n, X, dim, r, out_c, out_inter, static_cast<double*>(h->q_term.p), out_sum, st),
       "neighbourhood preservation");
    h->kernel_launches += 2;
    h->last_stream = st;
    return GUMAP_OK;
}

int gumap_quality_stress(gumap_knn* h, const float* X, int32_t dim, double* out_rows, double* out_stress,
                         void* stream) {
    if (!h) return fail(GUMAP_ERR_INVALID_ARG, "NULL handle");
    forget_runs(h);  // a captured run may not outlive this call (GUMAP_OPT_GRAPH)
    if (h->batch) return fail(GUMAP_ERR_INVALID_ARG, "quality metrics take a single graph's handle");
    if (!X || !out_stress) return fail(GUMAP_ERR_INVALID_ARG, "NULL drawing or output");
    if (dim < 1 || dim > 8) return fail(GUMAP_ERR_INVALID_ARG, "dim must be in [1, 8]");
    if (h->n > 65535) return fail(GUMAP_ERR_INVALID_ARG, "stress takes n <= 65535 (uint16 hop distances)");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    reap(h, false);
    const size_t n = (size_t)h->n;
    int rc;
    if ((rc = ensure(h, h->q_apsp, n * n * sizeof(uint16_t), "all-pairs rows")) ||
        (rc = ensure(h, h->q_idx, n * (size_t)h->k * sizeof(int32_t), "kNN rows")) ||
        (rc = ensure(h, h->q_dist, n * (size_t)h->k * sizeof(uint16_t), "kNN distances")) ||
        (!out_rows && (rc = ensure(h, h->q_term, n * sizeof(double), "stress rows"))))
        return rc;
    uint16_t* D = static_cast<uint16_t*>(h->q_apsp.p);
    double* rows = out_rows ? out_rows : static_cast<double*>(h->q_term.p);
    CK(cudaMemsetAsync(D, 0xFF, n * n * sizeof(uint16_t), st), "preset rows");
    if ((rc = run_msbfs(h, h->d_identity, true, h->n, static_cast<int32_t*>(h->q_idx.p),
                        static_cast<uint16_t*>(h->q_dist.p), st, D, true)))
        return rc;
    CK(launch_stress_rows(D, (long long)n, h->n, 0, h->n, X, dim, rows, st), "stress rows");
    CK(launch_sum(rows, (long long)n, 1.0 / ((double)n * (double)n - (double)n), out_stress, st), "stress sum");
    h->kernel_launches += 2;
    h->last_stream = st;
    return GUMAP_OK;
}

int gumap_spectral_layout(gumap_knn* h, int32_t dim, float* out_X, double* out_mu, gumap_spectral_info* info,
                          void* stream) {
    if (!h) return fail(GUMAP_ERR_INVALID_ARG, "NULL handle");
    forget_runs(h);  // a captured run may not outlive this call (GUMAP_OPT_GRAPH)
    if (!out_X) return fail(GUMAP_ERR_INVALID_ARG, "NULL output");
    if (dim < 1 || dim > 8) return fail(GUMAP_ERR_INVALID_ARG, "dim must be in [1, 8]");
    if (!h->last_union) return fail(GUMAP_ERR_INVALID_ARG, "the last run built no union COO");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    reap(h, false);
    const int32_t n = h->last_n_src;
    int rc;
    SpectralInput in{};
    in.n = n;
    if (h->coo_rows) {
        in.rowoff = h->coo.rowoff;
        in.col = h->coo.ccol;
        in.w = h->coo.cw;
    } else {
        unsigned long long nnz = 0;
        CK(cudaMemcpyAsync(&nnz, &h->d_ctr->coo_nnz, sizeof(nnz), cudaMemcpyDeviceToHost, st), "read nnz");
        CK(cudaStreamSynchronize(st), "read nnz");
        if ((rc = ensure(h, h->sp_rowoff, ((size_t)n + 1) * 8, "spectral rows")) ||
            (rc = ensure(h, h->sp_col, std::max<size_t>(nnz, 1) * 4, "spectral columns")))
            return rc;
        CK(launch_radix_csr(h->coo_keys, (long long)nnz, h->coo_key_bits, n,
                            static_cast<unsigned long long*>(h->sp_rowoff.p), static_cast<int32_t*>(h->sp_col.p), st),
           "spectral csr");
        in.rowoff = static_cast<unsigned long long*>(h->sp_rowoff.p);
        in.col = static_cast<int32_t*>(h->sp_col.p);
        in.w = h->coo_vals;
    }
    const size_t nn = (size_t)n;
    const long long by_memory = (long long)((4ull << 30) / (8ull * nn));
    const int m_max = (int)std::max<long long>(1, std::min<long long>({(long long)n - 1, 400ll, by_memory}));
    const size_t chunks = (nn + kSpectralChunk - 1) / kSpectralChunk;
    if ((rc = ensure(h, h->sp_vec, (5 + (size_t)dim) * nn * 8, "spectral vectors")) ||
        (rc = ensure(h, h->sp_Q, (size_t)m_max * nn * 8, "spectral basis")) ||
        (rc = ensure(h, h->sp_part, ((size_t)m_max + 1) * (chunks + 1) * 8, "spectral partial sums")))
        return rc;
    double* v = static_cast<double*>(h->sp_vec.p);
    SpectralScratch scr{};
    scr.s = v;
    scr.sq = v + nn;
    scr.t = v + 2 * nn;
    scr.w = v + 3 * nn;
    scr.z = v + 4 * nn;
    scr.Y = v + 5 * nn;
    scr.Q = static_cast<double*>(h->sp_Q.p);
    scr.part = static_cast<double*>(h->sp_part.p);
    scr.h = scr.part + ((size_t)m_max + 1) * chunks;
    scr.m_max = m_max;
    const int r = spectral_layout(in, dim, out_X, out_mu, info, scr, st);
    h->last_stream = st;
    if (r == -2) return fail(GUMAP_ERR_INVALID_ARG, "the union graph has no edge");
    if (r != 0) return cuda_fail(static_cast<cudaError_t>(r), "spectral layout");
    h->kernel_launches += 1;
    return GUMAP_OK;
}

int gumap_selftest_wait_timeout(int device, double limit_s) {
    if (!(limit_s >= 1e-3 && limit_s <= 5.0)) return fail(GUMAP_ERR_INVALID_ARG, "limit must be in [1 ms, 5 s]");
    CK(cudaSetDevice(device), "cudaSetDevice");
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device), "device attribute");
    void* buf = nullptr;
    CK(cudaMalloc(&buf, 64), "cudaMalloc");
    GridBarrier* bar = static_cast<GridBarrier*>(buf);
    int32_t* status = reinterpret_cast<int32_t*>(static_cast<char*>(buf) + 32);
    cudaError_t e = cudaMemset(buf, 0, 64);
    if (e == cudaSuccess)
        e = launch_barrier_selftest(bar, status, (unsigned long long)(limit_s * 1e9), sms, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int32_t st = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    return st == 0 ? fail(GUMAP_ERR_CUDA, "the bounded wait completed although it could not") : st;
}

int gumap_knn_rho_sigma(gumap_knn* h, float* rho, float* sigma, void* stream) {
    if (!h || h->last_n_src < 0) return fail(GUMAP_ERR_INVALID_ARG, "no run yet");
    if (h->last_n_src == 0) return GUMAP_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    if (rho) CK(cudaMemcpyAsync(rho, h->rho.p, (size_t)h->last_n_src * 4, cudaMemcpyDeviceToDevice, st), "copy rho");
    if (sigma) CK(cudaMemcpyAsync(sigma, h->sigma.p, (size_t)h->last_n_src * 4, cudaMemcpyDeviceToDevice, st), "copy sigma");
    h->last_stream = st;
    return GUMAP_OK;
}

int gumap_knn_coo(gumap_knn* h, int32_t* row, int32_t* col, float* w, int64_t* nnz, void* stream) {
    if (!h || !h->last_union) return fail(GUMAP_ERR_INVALID_ARG, "last run built no union COO");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const long long cap = 2ll * h->last_n_src * h->k;
    if (h->coo_rows) {
        CK(launch_coo_unpack(h->coo, cap, row, col, w, nnz, static_cast<cudaStream_t>(stream)), "coo unpack");
    } else {
        CK(launch_pairs_unpack(h->coo_keys, h->coo_vals, h->coo_key_bits, h->d_ctr, cap, row, col, w, nnz,
                               static_cast<cudaStream_t>(stream)),
           "coo unpack");
    }
    h->last_stream = static_cast<cudaStream_t>(stream);
    h->kernel_launches++;
    return GUMAP_OK;
}

int gumap_knn_check(gumap_knn* h, void* stream) {
    if (!h) return fail(GUMAP_ERR_INVALID_ARG, "NULL handle");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "stream sync");
    int32_t st = 0;
    CK(cudaMemcpy(&st, &h->d_ctr->status, sizeof(int32_t), cudaMemcpyDeviceToHost), "read status");
    if (st != 0) {
        CK(cudaMemset(&h->d_ctr->status, 0, sizeof(int32_t)), "clear status");
        return fail(st, "device reported %s", gumap_status_string(st));
    }
    return GUMAP_OK;
}

int gumap_knn_set_option(gumap_knn* h, int option, int64_t value) {
    if (!h) return fail(GUMAP_ERR_INVALID_ARG, "NULL handle");
    forget_runs(h);  // a captured run may not outlive this call (GUMAP_OPT_GRAPH)
    switch (option) {
        case GUMAP_OPT_ENGINE:
            if (value < GUMAP_ENGINE_AUTO || value > GUMAP_ENGINE_BATCH || value == GUMAP_ENGINE_MSBFS_SM)
                return fail(GUMAP_ERR_INVALID_ARG, "bad engine");
            if (value == GUMAP_ENGINE_BATCH && !h->batch && !h->batch_planned) {
                // a single graph as a one-graph batch (TOO_LARGE when it does not fit a CTA)
                CK(cudaSetDevice(h->device), "cudaSetDevice");
                CK(cudaDeviceSynchronize(), "sync");
                h->batch_offsets = {0, h->n};
                h->batch_modes = {h->mode};
                h->batch_edges = {h->nnz};
                if (int rc = apply_batch_plan(h, kMaxBatchW)) return rc;
            }
            if (value == GUMAP_ENGINE_FRONTIER && h->mode != GUMAP_PARTIAL)
                return fail(GUMAP_ERR_INVALID_ARG, "the frontier engine computes the partial form only");
            h->opt_engine = (int)value;
            return GUMAP_OK;
        case GUMAP_OPT_BLOCK_BITS:
            if (value < 0 || value % 128 != 0 || value > (1 << 20)) return fail(GUMAP_ERR_INVALID_ARG, "block bits must be a multiple of 128");
            h->opt_block_bits = value;
            return GUMAP_OK;
        case GUMAP_OPT_PROFILE:
            h->opt_profile = value ? 1 : 0;
            return GUMAP_OK;
        case GUMAP_OPT_STATE_BYTES:
            if (value < 0) return fail(GUMAP_ERR_INVALID_ARG, "negative budget");
            h->opt_state_bytes = value;
            return GUMAP_OK;
        case GUMAP_OPT_DIRECTION:
            if (value < 0 || value > 2) return fail(GUMAP_ERR_INVALID_ARG, "direction must be 0, 1 or 2");
            h->opt_direction = (int)value;
            return GUMAP_OK;
        case GUMAP_OPT_PULL_WIDTH:
            if (value != 2 && value != 4) return fail(GUMAP_ERR_INVALID_ARG, "pull width must be 2 or 4 words");
            h->opt_pull_width = (int)value;
            return GUMAP_OK;
        case GUMAP_OPT_BATCH_WIDTH:
            if (!h->batch && !h->batch_planned)
                return fail(GUMAP_ERR_INVALID_ARG, "batch width applies to batch handles and the batched engine");
            if (value < 0 || value > kMaxBatchW) return fail(GUMAP_ERR_INVALID_ARG, "batch width must be in [0, 64]");
            CK(cudaSetDevice(h->device), "cudaSetDevice");
            CK(cudaDeviceSynchronize(), "sync");
            return apply_batch_plan(h, value == 0 ? kMaxBatchW : (int32_t)value);
        case GUMAP_OPT_COO_BUILD:
            if (value < 0 || value > 2) return fail(GUMAP_ERR_INVALID_ARG, "COO build must be 0, 1 or 2");
            h->opt_coo_build = (int)value;
            return GUMAP_OK;
        case GUMAP_OPT_FRONTIER_BUILD:
            if (value < 0 || value > 3) return fail(GUMAP_ERR_INVALID_ARG, "frontier build must be 0, 1, 2 or 3");
            h->opt_frontier_build = (int)value;
            return GUMAP_OK;
        case GUMAP_OPT_GRAPH:
            if (value != 0 && value != 1) return fail(GUMAP_ERR_INVALID_ARG, "graph option must be 0 or 1");
            h->opt_graph = (int)value;
            return GUMAP_OK;
        case GUMAP_OPT_STAGE:
            if (value < 0 || value > 2) return fail(GUMAP_ERR_INVALID_ARG, "stage must be 0, 1 or 2");
            h->opt_stage = (int)value;
            return GUMAP_OK;
        case GUMAP_OPT_CTAS_PER_SM:
            if (value != 0 && value != 3 && value != 4) return fail(GUMAP_ERR_INVALID_ARG, "CTAs per SM must be 3 or 4");
            h->opt_ctas_per_sm = value == 4 ? 4 : 3;
            return GUMAP_OK;
        case GUMAP_OPT_PUSH_DIV:
            if (value < 1 || value > (1 << 20)) return fail(GUMAP_ERR_INVALID_ARG, "push divisor out of range");
            h->opt_push_div = (int)value;
            return GUMAP_OK;
        case GUMAP_OPT_HEAVY_DEGREE:
            if (value < 0 || value > 0x7FFFFFFF) return fail(GUMAP_ERR_INVALID_ARG, "bad degree threshold");
            CK(cudaSetDevice(h->device), "cudaSetDevice");
            CK(cudaDeviceSynchronize(), "sync");
            h->heavy_deg = (int32_t)value;
            if (int rc = build_order(h)) return rc;
            CK(cudaDeviceSynchronize(), "sync");  // the rows gathered on the legacy stream are ready for any stream
            return GUMAP_OK;
        default:
            return fail(GUMAP_ERR_INVALID_ARG, "unknown option %d", option);
    }
}

int gumap_knn_get_info(gumap_knn* h, gumap_knn_info* out) {
    if (!h || !out) return fail(GUMAP_ERR_INVALID_ARG, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->n = h->n;
    out->nnz = h->nnz;
    out->k = h->k;
    out->mode = h->mode;
    out->flags = h->flags;
    int32_t maxd = 0;
    for (int32_t d : h->deg) maxd = std::max(maxd, d);
    out->max_degree = maxd;
    out->batch = h->batch ? 1 : 0;
    return GUMAP_OK;
}

int gumap_knn_get_stats(gumap_knn* h, gumap_knn_stats* out) {
    if (!h || !out) return fail(GUMAP_ERR_INVALID_ARG, "NULL argument");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(cudaDeviceSynchronize(), "sync");
    DeviceCounters c;
    CK(cudaMemcpy(&c, h->d_ctr, sizeof(c), cudaMemcpyDeviceToHost), "read counters");
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->ev_pool[i], h->ev_pool[i + 1]) != cudaSuccess) continue;
        const int stage = h->ev_stage[i / 2];
        (stage == kStageSort ? h->sort_ms_done : stage == kStageWeights ? h->weights_ms_done : h->bfs_ms_done) += ms;
    }
    h->ev_used = 0;
    memset(out, 0, sizeof(*out));
    out->engine = h->last_engine;
    out->block_bits = h->last_block_bits;
    out->n_blocks = h->last_blocks;
    out->levels_max = c.levels_max;
    out->bfs_launches = h->bfs_launches;
    out->bfs_ms = h->bfs_ms_done;
    out->bfs_level_sum = c.level_sum;
    out->kernel_launches = h->kernel_launches;
    out->device_bytes = (int64_t)held_bytes(h);
    out->bfs_init_ms = (double)c.t_init_ns * 1e-6;
    out->bfs_pull_ms = (double)c.t_pull_ns * 1e-6;
    out->bfs_extract_ms = (double)c.t_extract_ns * 1e-6;
    out->bfs_push_ms = (double)c.t_push_ns * 1e-6;
    out->bfs_push_levels = c.push_levels;
    out->bfs_staged_launches = h->staged_launches;
    out->graph_replays = h->graph_replays;
    out->weights_ms = h->weights_ms_done;
    out->sort_ms = h->sort_ms_done;
    out->sort_launches = h->sort_launches;
    out->batch_model_bytes = (int64_t)c.model_bytes;
    return GUMAP_OK;
}

int gumap_knn_reset_stats(gumap_knn* h) {
    if (!h) return fail(GUMAP_ERR_INVALID_ARG, "NULL handle");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(cudaDeviceSynchronize(), "sync");
    h->bfs_launches = 0;
    h->kernel_launches = 0;
    h->staged_launches = 0;
    h->bfs_ms_done = 0.0;
    h->weights_ms_done = 0.0;
    h->sort_ms_done = 0.0;
    h->sort_launches = 0;
    h->graph_replays = 0;
    h->ev_used = 0;
    DeviceCounters c;
    CK(cudaMemcpy(&c, h->d_ctr, sizeof(c), cudaMemcpyDeviceToHost), "read counters");
    c.levels_max = 0;
    c.level_sum = 0;
    c.t_init_ns = c.t_pull_ns = c.t_extract_ns = c.t_push_ns = 0;
    c.push_levels = 0;
    c.model_bytes = 0;
    CK(cudaMemcpy(h->d_ctr, &c, sizeof(c), cudaMemcpyHostToDevice), "write counters");
    return GUMAP_OK;
}

}  // extern "C"
