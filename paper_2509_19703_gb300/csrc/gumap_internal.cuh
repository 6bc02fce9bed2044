// Internal declarations shared by the CUDA translation units of libgumap.
// Nothing here is part of the public ABI (include/gumap.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "gumap.h"

namespace gumap {

constexpr uint16_t kDistInf = 0xFFFFu;
constexpr int kMaxK = 256;
// A device-side wait that has not finished after this long gives up and
// reports GUMAP_ERR_TIMEOUT instead of hanging the GPU.
constexpr unsigned long long kWaitLimitNs = 10ull * 1000ull * 1000ull * 1000ull;

// Status values written by kernels into DeviceCounters::status.
constexpr int kStatusTimeout = 7;     // == GUMAP_ERR_TIMEOUT
constexpr int kStatusBadSource = 1;   // == GUMAP_ERR_INVALID_ARG (a source id outside [0, n))
constexpr int kStatusInternal = 4;    // == GUMAP_ERR_CUDA (device data disagrees with a host-side check)

struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};

// Small per-handle block of device counters; zeroed at handle creation. The
// fields before `status` belong to one MS-BFS launch: the host zeroes them
// (kLaunchCounterBytes) on the launch's stream before every launch.
struct DeviceCounters {
    GridBarrier bar;
    int32_t n_need;            // sources of the running block whose list is incomplete
    uint32_t lvl_any[3];       // "some vertex was reached at level d" in slot d % 3
    // direction choice of the MS-BFS levels (slot d % 4 belongs to level d)
    int32_t qcnt[4];                 // vertices in the frontier queue of level d
    int32_t qvalid[4];               // 1 if that queue was built
    unsigned long long f_edges[4];   // sum of deg(v) over nonzero (v, group) items of level d
    unsigned long long u_edges[4];   // sum of deg(v) over (v, group) items left unvisited after a pull
    // full form: (v, group) items all of whose active sources have reached v
    // after the pull of level d; when it is every item, level d + 1 is empty
    unsigned long long sat_items[4];
    uint32_t sat_seen;         // 1 once some pull item has had every active source reach it
    // ---- kept across launches
    int32_t status;
    int32_t levels;            // deepest level reached by the last MS-BFS launch
    int32_t levels_max;        // max over launches since the last host reset
    int32_t aux_count;         // scratch counter of the set-up kernels
    long long level_sum;       // sum of levels over launches since the last host reset
    unsigned long long coo_nnz;  // valid (key, value) pairs of the radix-sorted COO
    // device time of the MS-BFS phases (globaltimer ns, block 0's view at the
    // grid barriers), summed over launches since the last host reset
    unsigned long long t_init_ns;
    unsigned long long t_pull_ns;
    unsigned long long t_extract_ns;
    long long push_levels;           // push levels run since the last host reset
    unsigned long long t_push_ns;    // device time of push levels (prep + push)
    // batched engine: bytes of its units on the global engine's per-level
    // model (bitset streams plus CSR), summed since the last host reset
    unsigned long long model_bytes;
};
constexpr size_t kLaunchCounterBytes = offsetof(DeviceCounters, status);

// Arguments of one multi-source BFS launch over a block of sources.
struct MsbfsArgs {
    const int32_t* row_ptr;  // CSR (device, read-only during the launch)
    const int32_t* col;
    int32_t n;
    const int32_t* src;      // block's sources: vertex of bit j is src[j]
    int32_t identity;        // 1: src[j] == src_lo + j for every j (a range of consecutive vertices)
    int32_t src_lo;
    int32_t nb;              // sources in the block (<= 32 * W)
    int32_t W;               // 32-bit words per vertex row, multiple of 4
    uint32_t* F;             // frontier  [n][W]
    uint32_t* N;             // next      [n][W]
    uint32_t* S;             // seen      [n][W] (every level so far, the frontier included)
    // Processing order of the pull: vertices of degree above the heavy
    // threshold (one warp per item), then the rest (one thread per item),
    // each list by decreasing degree so the longest items start first.
    const int32_t* heavy;
    int32_t n_heavy;
    const int32_t* light;
    int32_t n_light;
    uint32_t* act;           // [W] bit j: source j still propagates
    uint32_t* need;          // [W] bit j: list of source j still incomplete
    int32_t* cnt;            // [nb] entries found so far
    int32_t* out_idx;        // [nb][k] rows of this block
    uint16_t* out_dist;      // [nb][k]
    int32_t k;
    int32_t partial;         // 1: stop each source once its list is complete
    // optional all-pairs output (full form): row j of the block at apsp + j * apsp_ld, uint16 hop
    // distances, preset to 0xFFFF by the host; NULL: not requested
    uint16_t* apsp;
    long long apsp_ld;
    DeviceCounters* ctr;
    // direction-optimising levels: 0 = choose per level, 1 = pull only,
    // 2 = push from level 2 on; queue/inq may be NULL only with 1
    int32_t direction;
    int32_t push_div;        // push when frontier edges * push_div < unvisited edges
    int32_t* queue;          // [4][n] frontier queues, slot d % 4
    int32_t* inq;            // [n] level at which the vertex last entered a queue
    int32_t pull_width;      // words per pull item: 4 (128 bits; also when 0) or 2 (64 bits)
    // per pull item (v, group), [n][W / pull_width] bytes, 16-byte padded, zeroed by the kernel:
    // 0 = active; 1 = every active source has reached it (permanent: S only grows, act only
    // shrinks), its N word was written 0 once; 2 = both N buffers hold 0 for it, so later pulls
    // skip it. NULL: no skipping.
    uint8_t* sat;
    int32_t ctas_per_sm;     // kernel build: 3 (also when 0) or 4 resident CTAs per SM
    // Staged pull (staged = 1): the rows of the light vertices in processing
    // order (ocol) with per-position (vertex, offset into ocol) pairs (meta:
    // n_light + 1 entries used, 2 more of padding; ocol has 4 ints of
    // padding), cut into one slice of positions per CTA, [slice[b],
    // slice[b + 1]). Each CTA bulk-copies its slice into shared memory once
    // per launch and reads every level's neighbour ids from there; the host
    // has checked that each slice fits stage_bytes. staged = 0: rows are
    // read from the global CSR.
    // Hub segments: a position whose vertex field is negative, ~(h *
    // kHubSegMax + s), is segment s of heavy vertex heavy[h] (its row entries
    // [s L, min((s + 1) L, deg)), L = hub_seg_len(deg)). hub_segments = 1 when
    // the layout holds them: the seen-set pull then runs the hubs from the
    // slices (each segment ORs its row into S_d with atomics, exact because
    // seen sets only grow) and the frontier scheme skips these positions and
    // runs its warp-wide heavy items.
    const int2* meta;
    const int32_t* ocol;
    const int32_t* slice;
    int32_t hub_segments;
    int32_t staged;          // 2: staged build reading the slice from global memory (the path
                             // taken when a copy does not complete; for tests)
    int32_t stage_bytes;     // dynamic shared memory of the launch (0 when not staged)
    // 1: pull from the seen sets (consecutive sources, pull-only levels):
    // S_d lives in buffer d % 3 of {F, N, S}; a level reads S_{d-1} (own row
    // and the neighbours' rows) and writes S_d = S_{d-1} | (OR of the
    // neighbours' S_{d-1} & act & ~S_{d-1}); level d's new pairs are
    // S_d & ~S_{d-1}. 0: the frontier scheme of the file comment of msbfs.cu.
    int32_t seen_only;
};

// Shared-memory bytes one CTA's staged slice takes (the kernel rounds the
// same way): the (vertex, offset) pairs of positions [p0, p1] from an even
// index, and the neighbour ids [c0, c1) from a multiple of 4, so both
// copies start and end on 16-byte boundaries.
// Hub segments of the staged layout (see MsbfsArgs::meta): at most
// kHubSegMax per hub, each of at least 16 row entries.
constexpr int kHubSegMax = 4096;
__host__ __device__ inline int hub_seg_len(int deg) {
    const int l = (deg + kHubSegMax - 1) / kHubSegMax;
    return l < 16 ? 16 : l;
}
__host__ __device__ inline int hub_seg_count(int deg) {
    const int l = hub_seg_len(deg);
    return (deg + l - 1) / l;
}

inline long long stage_slice_bytes(long long p0, long long p1, long long c0, long long c1) {
    const long long m = (((p1 + 2) & ~1ll) - (p0 & ~1ll)) * 8;
    const long long c = (((c1 + 3) & ~3ll) - (c0 & ~3ll)) * 4;
    return m + c;
}

// Arguments of one partial-BFS launch with one warp per source.
struct FrontierArgs {
    const int32_t* row_ptr;
    const int32_t* col;
    int32_t n;
    const int32_t* src;      // NULL = identity
    int32_t n_src;
    int32_t k;
    int32_t* out_idx;
    uint16_t* out_dist;
    int32_t* status;         // set to kStatusBadSource for a source outside [0, n)
    int32_t build;           // GUMAP_OPT_FRONTIER_BUILD: 0 automatic (3), 1 thread, 2 warp, 3 group of lanes per source
    int32_t sms;             // SMs the launch may fill (its grid is sized for that many); 0 = all
};

// One unit of the batched engine: a block of sources of one graph of the
// batch (a disjoint union; the graph occupies vertices [v0, v0 + n)).
constexpr int kMaxBatchW = 64;  // at most 64 words (2048 sources) per unit
struct BatchUnit {
    int32_t v0;        // first vertex of the graph
    int32_t n;         // vertices of the graph
    int32_t s_lo;      // first source of the unit (graph-local id)
    int32_t nb;        // sources in the unit (<= 32 * W)
    int32_t W;         // words per bitset row
    int32_t partial;   // 1: partial form for this graph
    int32_t v_global;  // 1: visited bitset in the CTA's global slab
    int32_t pad;
};

struct BatchArgs {
    const int32_t* row_ptr;  // CSR of the disjoint union (global ids)
    const int32_t* col;
    const BatchUnit* units;
    int32_t n_units;
    int32_t k;
    int32_t* out_idx;        // [N][k], row = global vertex id
    uint16_t* out_dist;
    uint32_t* vslab;         // per CTA: vslab + blockIdx.x * vslab_words
    long long vslab_words;
    int32_t* next_unit;      // work-queue counter, zeroed before the launch
    DeviceCounters* ctr;
};

// Shared-memory bytes a batched unit may use (the rest of the 227 KB holds
// the kernel's static shared arrays).
constexpr size_t kBatchSmemBudget = 220000;

// ---- gumap_capi.cu (host helpers shared with the server)
// Sets the calling thread's gumap_last_error() message; returns status.
int report_error(int status, const char* msg);
bool host_csr_ok(const int32_t* rp, const int32_t* col, int32_t n, int64_t nnz, std::string& why);
// graph_edges[g]: adjacency entries of graph g; max_w: widest unit allowed (words, <= kMaxBatchW).
int32_t plan_batch(int32_t n_graphs, const int32_t* vertex_offsets, const int64_t* graph_edges, const int32_t* modes,
                   std::vector<BatchUnit>& units, size_t& smem, long long& slab, int32_t max_w = kMaxBatchW);

// ---- pool.cu: the handles' device-memory pool, and the SM count of the current device
// (queried once per device; grid caps are multiples of it)
int device_sm_count();
cudaError_t pool_alloc(void** p, size_t bytes);
void pool_free(void* p, size_t bytes);  // the device must be done with p
void pool_trim(int device);             // device < 0: every device
size_t pool_cached_bytes();

// ---- tune.cu
void tune_apply_cached(struct gumap_knn* h, const char* cache_path);

// ---- batch.cu
cudaError_t batch_prepare(size_t smem_bytes);
int batch_threads();
const void* batch_kernel_ptr();
cudaError_t launch_batch(const BatchArgs& a, int grid, size_t smem_bytes, cudaStream_t s);

// ---- msbfs.cu
int msbfs_max_blocks_per_sm(int block_threads, int pull_width = 4, int ctas_per_sm = 3, size_t dyn_smem = 0,
                            bool staged = false);
// Allows the kernel builds up to `bytes` of dynamic shared memory.
cudaError_t msbfs_allow_smem(int bytes);
cudaError_t launch_gather_rows(const int32_t* row_ptr, const int32_t* col, const int32_t* heavy, const int2* meta,
                               int32_t n_pos,
                               int32_t* ocol, cudaStream_t s);
cudaError_t launch_msbfs(const MsbfsArgs& a, int grid, int block, cudaStream_t s);
int msbfs_grid_for(const MsbfsArgs& a, int max_grid);
cudaError_t launch_identity(int32_t* dst, int32_t n, cudaStream_t s);
cudaError_t launch_barrier_selftest(GridBarrier* bar, int32_t* status, unsigned long long limit_ns, int grid,
                                    cudaStream_t s);

// ---- frontier.cu
cudaError_t launch_frontier(const FrontierArgs& a, cudaStream_t s);

// ---- weights.cu
// Per-row record of the smoothing step (16 bytes, one aligned load): the key
// of the row's last list slot (its id and distance; last_dist = kDistInf and
// last_id = -1 when the list is padded, i.e. holds every vertex the row's
// vertex reaches), and the row's rho and sigma. The union reads it to decide
// whether a row lists a given vertex and to recompute that slot's weight.
struct __align__(16) WeightRow {
    int32_t last_id;
    int32_t last_dist;
    int32_t rho;
    float sigma;
};
// Dynamic shared memory of one smoothing launch for k slots per row.
size_t smooth_knn_smem_bytes(int32_t k);
// rho, sigma [n_rows]; rec (NULL: not written; needs idx) [n_rows]; a (NULL:
// not written) the directed weights [n_rows][k]. Rows: distances ascending,
// padding 0xFFFF last, as every engine writes them.
cudaError_t launch_smooth_knn(const int32_t* idx, const uint16_t* dist, int32_t n_rows, int32_t k, float T,
                              float* rho, float* sigma, WeightRow* rec, float* a, cudaStream_t s);
// Union weights into w from the lists and the records.
cudaError_t launch_union(const int32_t* idx, const uint16_t* dist, const WeightRow* rec, int32_t n, int32_t k,
                         float* w, cudaStream_t s);
// Look-back state of the union's mirror compaction: one published word per
// tile of slots (union_scan_words of them) and a tile counter, both zeroed;
// the mirror total lands in *total.
struct UnionScan {
    unsigned long long* pub;
    unsigned int* tile_ctr;
    unsigned long long* total;
    int32_t* status;                 // kStatusTimeout if a look-back wait gives up
    unsigned long long limit_ns;
};
size_t union_scan_words(int32_t n, int32_t k);
// Union weights into w, per row the valid-slot count (kval), and the mirrors
// (slots whose target does not list the row) compacted in slot order as keys
// (i << 32) | j with the slot's weight.
cudaError_t launch_union_mirrors(const int32_t* idx, const uint16_t* dist, const WeightRow* rec, int32_t n,
                                 int32_t k, float* w, int32_t* kval, unsigned long long* mkey, float* mval,
                                 const UnionScan& scan, cudaStream_t s);

// Below kCooRowsMinSlots slots the COO is 2 n k (key, value) pairs sorted by
// the radix sort; the row-by-row build's long-row tails cost more there than
// the passes it saves.
constexpr long long kCooRowsMinSlots = 2ll << 20;
// Union weights into w and the 2 * n * k COO (key, value) pairs (padding
// pairs all ones), counting the valid pairs into ctr->coo_nnz.
cudaError_t launch_union_pairs(const int32_t* idx, const uint16_t* dist, const WeightRow* rec, int32_t n, int32_t k,
                               float* w, int key_bits, unsigned long long* keys, float* vals, DeviceCounters* ctr,
                               cudaStream_t s);
cudaError_t launch_pairs_unpack(const unsigned long long* keys, const float* vals, int key_bits,
                                const DeviceCounters* ctr, long long cap, int32_t* row, int32_t* col, float* w,
                                int64_t* nnz_out, cudaStream_t s);

// ---- sort.cu: LSD radix sort of (u64 key, float value) on the low `bits` key bits
// (bits <= 64). A look-back wait that gives up writes kStatusTimeout to *status.
// count_dev (optional): the element count on the device, at most `count`
// (which then only bounds the launch).
size_t radix_sort_temp_bytes(long long count, int bits);
cudaError_t radix_sort_pairs(unsigned long long* keys, float* vals, unsigned long long* keys_tmp,
                             float* vals_tmp, long long count, int bits, void* temp, size_t temp_bytes,
                             int32_t* status, cudaStream_t s, unsigned long long** keys_out, float** vals_out,
                             int* launches, const unsigned long long* count_dev = nullptr);

// ---- coo.cu: the fuzzy union as a COO sorted by (row, col), built by rows
constexpr int kCooCtrTile = 0;               // tile counter of the row scan
constexpr int kCooCtrWords = 4;

struct CooArgs {
    const int32_t* idx;          // kNN lists [n][k], valid slots first
    const float* w;              // union weight per slot [n][k]
    const int32_t* kval;         // per row: valid slots (own entries)
    int32_t n;
    int32_t k;
    // the mirrors sorted by target, stably (so by source within a target):
    // key (source << 32) | target, value the slot's weight; how many there
    // are is on the device (*mirrors), at most n k
    const unsigned long long* tkey;
    const float* tval;
    const unsigned long long* mirrors;
    int32_t key_bits;            // the target's bits in a key: 2^key_bits > n
    uint32_t* instart;           // [n] first sorted mirror of each target (zeroed)
    uint32_t* inend;             // [n] one past its last (zeroed): mirrors of row i = inend - instart
    uint32_t* mcnt;              // [n] mirrors per row
    int32_t* scol;               // [n][k] own entries sorted by column
    float* sw;                   // their weights
    unsigned long long* rowoff;  // [n + 1] first entry of each row; rowoff[n] = nnz
    unsigned long long* pub;     // look-back words of the row scan [tiles], zeroed
    uint32_t* ctr;               // [kCooCtrWords], zeroed
    int32_t* ccol;               // the COO rows [<= 2 n k]: columns ascending in each row
    float* cw;
    int32_t* status;             // kStatusTimeout if a look-back wait gives up
};
// One zeroed block per run: instart, inend (each [n], 16-byte padded), ctr, pub.
size_t coo_scratch_bytes(int32_t n);
void coo_scratch_split(void* scratch, int32_t n, uint32_t** instart, uint32_t** inend, uint32_t** ctr,
                       unsigned long long** pub);
// After launch_union_mirrors and the stable sort of the mirrors: target
// ranges, own-row sort, row scan, own entries, mirrors (5 launches).
cudaError_t launch_coo_build(const CooArgs& a, int sms, cudaStream_t s, int* launches);
// Rows, columns and weights of the sorted COO (up to cap entries) and nnz.
cudaError_t launch_coo_unpack(const CooArgs& a, long long cap, int32_t* row, int32_t* col, float* w,
                              int64_t* nnz_out, cudaStream_t s);

// ---- quality.cu: quality metrics of a drawing (Section 4.1.3)
// Neighbourhood preservation: per vertex |N_G(v, r)| (out_c) and |N_G cap N_D|
// (out_inter), both optional; term [n] receives each vertex's Jaccard term;
// *out_sum their sum.
cudaError_t launch_np(const int32_t* row_ptr, const int32_t* col, int32_t n, const float* X, int32_t dim, int32_t r,
                      int32_t* out_c, int32_t* out_inter, double* term, double* out_sum, cudaStream_t s);
// Stress terms of `rows` all-pairs rows (row q is source src_lo + q, leading dimension ld) summed per row.
cudaError_t launch_stress_rows(const uint16_t* D, long long ld, int32_t rows, int32_t src_lo, int32_t n,
                               const float* X, int32_t dim, double* out_rows, cudaStream_t s);
// *out = scale * sum of vals[0 .. count), in a fixed order.
cudaError_t launch_sum(const double* vals, long long count, double scale, double* out, cudaStream_t s);

// ---- spectral.cu: spectral layout of the union graph (the layout stage's initial coordinates)
struct SpectralInput {
    const unsigned long long* rowoff;  // CSR of the symmetric weighted graph, [n + 1]
    const int32_t* col;
    const float* w;
    int32_t n;
};
struct SpectralScratch {
    double *s, *sq, *t, *w, *z;  // [n] each
    double* Q;                   // [m_max][n] Lanczos basis
    double* Y;                   // [dim][n] Ritz vectors
    double* part;                // [(m_max + 1) * ceil(n / 4096)] partial sums
    double* h;                   // [m_max + 1]
    int32_t m_max;
};
constexpr int kSpectralChunk = 4096;
// Returns 0, a cudaError_t value (> 0), or -2 when the graph has no edge. Synchronous on st.
int spectral_layout(const SpectralInput& in, int dim, float* out_X, double* out_mu, gumap_spectral_info* info,
                    SpectralScratch& scr, cudaStream_t st);
// rowoff [n + 1] and col [nnz] of the COO whose sorted keys are (row << key_bits) | col.
cudaError_t launch_radix_csr(const unsigned long long* keys, long long nnz, int key_bits, int32_t n,
                             unsigned long long* rowoff, int32_t* col, cudaStream_t s);

// ---- validate.cu
// Device-side CSR validation; writes 0 to *bad if the graph is valid.
cudaError_t launch_validate_csr(const int32_t* row_ptr, const int32_t* col, int32_t n, int64_t nnz,
                                int32_t* bad, cudaStream_t s);

}  // namespace gumap
