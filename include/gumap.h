/*
 * gumap.h - C ABI of the GB300 graph-kNN library.
 *
 * The library computes, for an undirected unweighted graph G = (V, E) and a
 * neighbourhood size k, the graph-theoretic kNN graph used by UMAP-based
 * graph drawing, and the UMAP fuzzy weights of its edges:
 *
 *   C0  hop distances by breadth-first search from each source vertex,
 *       either to completion (the all-pairs distances of GUMAP, Algorithm 1)
 *       or stopped once k other vertices are reached (the partial BFS of
 *       SL-GUMAP, Algorithm 4, Section 3.3.1);
 *   C1  the k nearest other vertices of each source in (distance, vertex id)
 *       order (Algorithm 1, its kNN step; the paper breaks ties at random, this
 *       library fixes the tie rule to ascending vertex id so the result is
 *       unique and identical between the two forms);
 *   W   rho_i = distance to the nearest neighbour, sigma_i solving
 *       sum_j exp(-max(0, d_ij - rho_i) / sigma_i) = log2 k, and the directed
 *       similarity a_ij = exp(-max(0, d_ij - rho_i) / sigma_i) (Section 2.1,
 *       h_ij), then the fuzzy union w_ij = a_ij + a_ji - a_ij a_ji of the
 *       UMAP implementation the paper builds on (Section 4.1.1).
 *
 * Conventions shared by every call:
 *   - Vertex ids are int32 in [0, n). Distances are hop counts stored as
 *     uint16; GUMAP_DIST_INF (0xFFFF) marks a padded slot.
 *   - A source with fewer than k reachable other vertices gets its reachable
 *     ones followed by padding: id -1, distance 0xFFFF, weight 0 (Section 3.2:
 *     pairs with no connecting path carry an "infinite" value).
 *   - Every call returns an int status (GUMAP_OK = 0). Nothing throws or
 *     aborts across the ABI. gumap_status_string() names a status;
 *     gumap_last_error() returns a message for the calling thread's last
 *     failure.
 *   - "device" pointers are CUDA device (or managed) memory of the handle's
 *     device; "host" pointers are ordinary CPU memory.
 *   - A gumap_knn handle is not thread-safe: one thread (or external locking)
 *     per handle. Different handles may be used concurrently.
 *   - Work is enqueued on the caller's cudaStream_t passed as `void* stream`
 *     (NULL = the legacy default stream). Calls marked "asynchronous" return
 *     before the device work finishes; their outputs are valid once the
 *     stream reaches that point.
 */
#ifndef GUMAP_H
#define GUMAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define GUMAP_OK                  0
#define GUMAP_ERR_INVALID_ARG     1  /* a pointer, size, k, mode or flag is invalid */
#define GUMAP_ERR_INVALID_GRAPH   2  /* CSR not symmetric / unsorted / self loop / duplicate / id out of range */
#define GUMAP_ERR_OOM             3  /* device or host allocation failed */
#define GUMAP_ERR_CUDA            4  /* a CUDA runtime call failed (see gumap_last_error) */
#define GUMAP_ERR_AGAIN           5  /* server queue full: retry later */
#define GUMAP_PENDING             6  /* server request not finished yet */
#define GUMAP_ERR_TIMEOUT         7  /* a bounded device-side wait gave up (no hang, no trap) */
#define GUMAP_ERR_TOO_LARGE       8  /* request can never fit the server's device-memory budget */
#define GUMAP_ERR_UNKNOWN_REQUEST 9  /* server request id unknown or already released */

/* ------------------------------------------------------------------ modes */
#define GUMAP_FULL    0  /* BFS to completion from each source (GUMAP, Algorithm 1) */
#define GUMAP_PARTIAL 1  /* BFS stopped at the level that reaches k (SL-GUMAP, Algorithm 4) */

/* ------------------------------------------------------------------ flags */
#define GUMAP_WEIGHTS_UNION    0x0u /* out_w = fuzzy-union weight w_ij (default; sources must be NULL) */
#define GUMAP_WEIGHTS_DIRECTED 0x1u /* out_w = directed similarity a_ij of the source's own list */
#define GUMAP_CSR_ON_DEVICE    0x2u /* row_ptr / col_idx passed to gumap_knn_create are device pointers */
#define GUMAP_EMIT_APSP        0x4u /* full form only: the handle may also emit all-pairs distance rows
                                       (gumap_knn_apsp)                                              */

#define GUMAP_MAX_K    256
#define GUMAP_DIST_INF 0xFFFFu

/* ---------------------------------------------------------------- engines */
#define GUMAP_ENGINE_AUTO     0 /* pick by graph size, mode and the tuned table */
#define GUMAP_ENGINE_MSBFS    1 /* bit-parallel multi-source BFS, bitsets in global memory (L2) */
#define GUMAP_ENGINE_MSBFS_SM 2 /* reserved, not accepted (small graphs in shared memory: GUMAP_ENGINE_BATCH) */
#define GUMAP_ENGINE_FRONTIER 3 /* partial form only: warp per source, bounded merge of sorted rows */
#define GUMAP_ENGINE_BATCH    4 /* one persistent launch, one CTA per (graph, source block), bitsets in
                                   shared memory: batch handles, and single graphs small enough for a
                                   CTA (selecting it for one graph plans a one-graph batch, which
                                   synchronises; TOO_LARGE beyond about 27,000 vertices); a run with
                                   explicit sources uses GUMAP_ENGINE_MSBFS instead                */

/* --------------------------------------------------------------- options */
#define GUMAP_OPT_ENGINE      1 /* value: GUMAP_ENGINE_*                                 */
#define GUMAP_OPT_BLOCK_BITS  2 /* value: sources per MS-BFS block (multiple of 128), 0 = auto */
#define GUMAP_OPT_PROFILE     3 /* value: 1 = time each BFS launch, the weights and the COO build with CUDA events */
#define GUMAP_OPT_STATE_BYTES 4 /* value: device bytes allowed for MS-BFS bitsets, 0 = auto */
#define GUMAP_OPT_HEAVY_DEGREE 5 /* value: MS-BFS vertices of larger degree are processed by a whole warp
                                    (default max(64, 4 x mean degree)); setting it synchronises the device */
#define GUMAP_OPT_DIRECTION   6 /* value: MS-BFS level direction: 0 = choose per level,
                                   1 = pull only (default), 2 = push from level 2 on            */
#define GUMAP_OPT_PUSH_DIV    7 /* value: push when frontier edges * value < unvisited edges (default 8) */
#define GUMAP_OPT_PULL_WIDTH  8 /* value: 32-bit words per MS-BFS pull item, 4 (default) or 2     */
#define GUMAP_OPT_CTAS_PER_SM 9 /* value: resident 256-thread MS-BFS CTAs per SM the kernel is built
                                   for: 3 (default, up to 80 registers a thread) or 4 (64)        */
#define GUMAP_OPT_BATCH_WIDTH 11 /* value: batched engine: widest unit in 32-bit words (32 sources each),
                                   1..64, 0 = 64 (default); re-plans the batch, synchronises      */
#define GUMAP_OPT_COO_BUILD  12 /* value: how gumap_knn_run builds the union COO: 0 = automatic (default:
                                   1 below 2^21 slots n x k, 2 from there on), 1 = LSD radix sort of
                                   2 n k (row, col) keys, 2 = row by row (the mirror entries, sorted
                                   stably by target, give each row's mirrors in id order; each row's
                                   own entries ranked by column; one scan; every entry placed by
                                   counting); same COO either way                                  */
#define GUMAP_OPT_FRONTIER_BUILD 13 /* value: the frontier engine's merge (partial form): 0 = automatic
                                   (default: groups of lanes), 1 = one thread per source (k <= 64;
                                   larger k use a warp), 2 = one warp per source, 3 = a group of
                                   4 to 32 lanes per source (by k); same rows either way          */
#define GUMAP_OPT_GRAPH      14 /* value: 1 = once two runs in a row had the same sources, outputs and
                                   (non-default) stream, the third is captured into a CUDA graph
                                   and every later run with those arguments replays it (one launch
                                   of the graph instead of one per kernel); any other call on the
                                   handle drops the graph; a capture the driver refuses falls back
                                   to ordinary launches; not with GUMAP_OPT_PROFILE. 0 (default) =
                                   ordinary launches                                              */
#define GUMAP_OPT_STAGE      10 /* value: 1 (default) = each MS-BFS CTA bulk-copies its slice of the
                                   ordinary-degree rows into shared memory once per launch when
                                   every slice fits; 0 = neighbour ids always read from the CSR;
                                   2 = (tests) the staged kernel reads its slice from global memory,
                                   the path it takes when a bulk copy does not complete           */

typedef struct gumap_knn gumap_knn;

/*
 * gumap_knn_create - validate and take a copy of a graph (the input graph of
 * Algorithm 1 and Algorithm 4).
 *
 *   h        out: new handle (NULL on failure).
 *   row_ptr  CSR row offsets, int32[n + 1], row_ptr[0] = 0, row_ptr[n] = nnz.
 *   col_idx  CSR column ids, int32[nnz]. The graph must be undirected and
 *            simple: every row sorted strictly ascending (no duplicates), no
 *            self loop, ids in [0, n), and (u, v) present iff (v, u) present.
 *   n        number of vertices, 1 <= n < 2^31.
 *   nnz      number of directed entries (2 |E|), 0 <= nnz < 2^31.
 *   k        neighbourhood size, 1 <= k <= min(n - 1, GUMAP_MAX_K) (k = 1 if n = 1 is rejected).
 *   mode     GUMAP_FULL or GUMAP_PARTIAL.
 *   flags    GUMAP_WEIGHTS_* | GUMAP_CSR_ON_DEVICE | GUMAP_EMIT_APSP (full form only).
 *   device   CUDA device ordinal; it becomes current on the calling thread.
 *
 * Host CSR (default) is validated on the host; device CSR is validated by a
 * device kernel before being copied (the call synchronises once). The
 * library copies the CSR into memory it owns; the caller's arrays may be
 * freed on return. Errors: INVALID_ARG, INVALID_GRAPH, OOM, CUDA.
 */
int gumap_knn_create(gumap_knn **h, const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                     int64_t nnz, int32_t k, int mode, uint32_t flags, int device);

/*
 * gumap_batch_create - one handle over many independent graphs, run in one
 * persistent launch (the method of Algorithm 1 / Algorithm 4 applied to each
 * graph; the graphs are laid side by side as a disjoint union).
 *
 *   n_graphs        number of graphs, >= 1.
 *   vertex_offsets  host int32[n_graphs + 1]: graph g owns vertices
 *                   [vertex_offsets[g], vertex_offsets[g + 1]) of the union;
 *                   vertex_offsets[0] = 0, strictly increasing (no empty graph).
 *   row_ptr,col_idx host CSR of the union with global ids (every rule of
 *                   gumap_knn_create, and no edge between two graphs).
 *   k               1 <= k <= min(N - 1, GUMAP_MAX_K), N = vertex_offsets[n_graphs];
 *                   a graph with fewer than k + 1 vertices gets padded rows.
 *   modes           host int32[n_graphs]: GUMAP_FULL or GUMAP_PARTIAL per graph.
 *   flags           GUMAP_WEIGHTS_* (the CSR must be on the host).
 *
 * gumap_knn_run(h, NULL, N, ...) then writes the rows of every vertex of
 * every graph (row = global vertex id; neighbour ids are global ids), the
 * weights and, for union weights, the COO of the union (each graph's COO is
 * a contiguous run). Each graph's rows are identical to what a handle of
 * that graph alone produces (after shifting ids). A graph must fit the
 * engine's per-CTA shared memory (about 27,000 vertices); larger graphs get
 * GUMAP_ERR_TOO_LARGE and belong in their own handle. The call synchronises
 * once. Errors: INVALID_ARG, INVALID_GRAPH, TOO_LARGE, OOM, CUDA.
 */
int gumap_batch_create(gumap_knn **h, int32_t n_graphs, const int32_t *vertex_offsets, const int32_t *row_ptr,
                       const int32_t *col_idx, int64_t nnz, int32_t k, const int32_t *modes, uint32_t flags,
                       int device);

/*
 * gumap_knn_run - compute the kNN lists and weights of a set of sources
 * (C0 + C1 + weights: the distance and kNN steps of Algorithm 1, or
 * Algorithm 4; Section 2.1). Asynchronous on `stream`.
 *
 *   sources  device int32[n_src] of source vertex ids, or NULL for all
 *            vertices 0..n-1 in order (then n_src must equal n).
 *   n_src    number of sources, 0 <= n_src <= 2^31 - 1.
 *   out_idx  device int32[n_src][k], row-major: row i lists the neighbours of
 *            sources[i] in (distance, id) order, padded with -1.
 *   out_dist device uint16[n_src][k]: hop distance of each slot, 0xFFFF pad.
 *   out_w    device float[n_src][k]: the union weight w_ij (GUMAP_WEIGHTS_UNION,
 *            requires sources == NULL) or the directed a_ij
 *            (GUMAP_WEIGHTS_DIRECTED); 0 for padded slots.
 *
 * All three outputs are owned by the caller and must not overlap. The call
 * grows library-owned scratch when n_src exceeds every earlier call, without
 * synchronising: a replaced block returns to the library's pool once the
 * work queued before it has finished. A handle's calls must be ordered on
 * the device (one stream, or streams the caller orders), since they share
 * the handle's scratch. With union weights the symmetric COO is
 * also built and kept in the handle for gumap_knn_coo(): below 2^21 slots
 * (n k) by an LSD radix sort of 2 n k (row, col) keys, from there on row by
 * row (GUMAP_OPT_COO_BUILD overrides the choice). The handle keeps that
 * build's scratch: about 48 n k bytes for the radix sort (keys and values,
 * twice), about 52 n k bytes for the row build. Errors:
 * INVALID_ARG (bad pointer/size, union with explicit sources), OOM, CUDA.
 * Device-side failures (a bounded wait that timed out) are reported by
 * gumap_knn_check().
 */
int gumap_knn_run(gumap_knn *h, const int32_t *sources, int32_t n_src, int32_t *out_idx,
                  uint16_t *out_dist, float *out_w, void *stream);

/*
 * gumap_knn_apsp - the hop distance from each source to every vertex: the
 * rows of the all-pairs shortest-path matrix S of Algorithm 1 (its C0 step;
 * here row by row for the given sources),
 * from the same bit-parallel BFS run to completion, together with the
 * source's kNN list as gumap_knn_run writes it (no weights are computed).
 * The handle must have been created with GUMAP_EMIT_APSP (full form).
 *
 *   sources   device int32[n_src], or NULL for all n vertices (n_src == n)
 *   out_idx   device int32[n_src][k], out_dist device uint16[n_src][k]: as gumap_knn_run
 *   out_apsp  device uint16[n_src][n], row i for source i: 0 at the source, hop distances,
 *             0xFFFF for vertices the source cannot reach (n must be at most 65535, so every
 *             distance fits below 0xFFFF: INVALID_ARG otherwise)
 *
 * Asynchronous on `stream`; rows are written in place (caller-owned).
 * Errors: INVALID_ARG (flag missing, NULL output, bad sources), OOM, CUDA;
 * device-side errors via gumap_knn_check().
 */
int gumap_knn_apsp(gumap_knn *h, const int32_t *sources, int32_t n_src, int32_t *out_idx, uint16_t *out_dist,
                   uint16_t *out_apsp, void *stream);

/*
 * gumap_knn_rho_sigma - copy rho_i and sigma_i of the last run (Section 2.1)
 * into device float[n_src] buffers. Asynchronous on `stream` (use the run's
 * stream or order it after). sigma is +inf for a row whose valid entries
 * number at most log2 k (every weight 1) and 0 for a row with no valid entry.
 * Errors: INVALID_ARG (no run yet, NULL pointer).
 */
int gumap_knn_rho_sigma(gumap_knn *h, float *rho, float *sigma, void *stream);

/*
 * gumap_knn_coo - copy the symmetric fuzzy-union graph of the last run as a
 * COO sorted by (row, col) (the union of Section 4.1.1's UMAP
 * implementation; every pair appears once, w_ij = w_ji).
 *
 *   row, col  device int32[2 * n * k] (capacity bound; may be NULL to skip)
 *   w         device float[2 * n * k] (may be NULL to skip)
 *   nnz       device int64[1]: receives the entry count, nk_valid <= nnz <= 2 nk_valid.
 *
 * Asynchronous on `stream`. Errors: INVALID_ARG (last run had no union).
 */
int gumap_knn_coo(gumap_knn *h, int32_t *row, int32_t *col, float *w, int64_t *nnz, void *stream);

/*
 * gumap_knn_check - wait for `stream` and report the device status word of
 * the handle's kernels: GUMAP_OK or GUMAP_ERR_TIMEOUT (a bounded device
 * barrier gave up; the outputs of that run are undefined, the context
 * stays usable). Clears the word.
 */
int gumap_knn_check(gumap_knn *h, void *stream);

/* gumap_knn_set_option - set a GUMAP_OPT_* value (takes effect on the next run). */
int gumap_knn_set_option(gumap_knn *h, int option, int64_t value);

typedef struct {
    int32_t engine;          /* GUMAP_ENGINE_* used by the last run */
    int32_t block_bits;      /* sources per MS-BFS block in the last run (0 if none) */
    int32_t n_blocks;        /* MS-BFS launches (source blocks) in the last run */
    int32_t levels_max;      /* deepest BFS level over the blocks of the last run */
    int64_t bfs_launches;    /* BFS kernel launches since the last reset */
    double  bfs_ms;          /* summed device time of those launches (GUMAP_OPT_PROFILE on), ms */
    int64_t bfs_level_sum;   /* sum over launches of the BFS levels each ran */
    int64_t kernel_launches; /* all library kernel launches since the last reset */
    int64_t device_bytes;    /* device memory held by the handle */
    double  bfs_init_ms;     /* MS-BFS device time in clearing + level-1 push (device timer) */
    double  bfs_pull_ms;     /* MS-BFS device time in the pull steps of levels >= 2 */
    double  bfs_extract_ms;  /* MS-BFS device time in the kNN extraction steps */
    double  bfs_push_ms;     /* MS-BFS device time in push levels (queue preparation + push) */
    int64_t bfs_push_levels; /* MS-BFS levels run as a push since the last reset */
    int64_t bfs_staged_launches; /* MS-BFS launches whose rows were staged in shared memory */
    double  weights_ms;      /* device time of rho/sigma, weights and union (GUMAP_OPT_PROFILE on), ms */
    double  sort_ms;         /* device time of the COO build, radix sort or rows (GUMAP_OPT_PROFILE on), ms */
    int64_t sort_launches;   /* COO build kernel launches since the last reset */
    int64_t batch_model_bytes; /* batched engine: its units' bytes on the per-level model of the
                                  bit-parallel BFS (3 bitset rows of n x W words, in shared memory
                                  there, plus the CSR, per level), since the last reset */
    int64_t graph_replays;   /* runs served by replaying a captured CUDA graph (GUMAP_OPT_GRAPH) */
} gumap_knn_stats;

typedef struct {
    int32_t n;
    int64_t nnz;
    int32_t k;
    int32_t mode;
    uint32_t flags;
    int32_t max_degree;
    int32_t batch;           /* 1 for handles made by gumap_batch_create */
} gumap_knn_info;

/* gumap_knn_get_info - the shape of the handle's graph and request. */
int gumap_knn_get_info(gumap_knn *h, gumap_knn_info *out);

typedef struct {
    int32_t from_cache;      /* 1: settings read from the cache, nothing timed */
    int32_t candidates;      /* settings timed */
    double best_ms;          /* device time of one gumap_knn_run with the chosen settings */
    double default_ms;       /* ... with the settings the handle had before */
    int32_t engine, pull_width, heavy_mult, direction;
    int64_t state_bytes;
    int32_t ctas_per_sm;
    int32_t stage;
    int32_t push_div;        /* push threshold of the automatic direction (when direction == 0) */
    int32_t batch_width;     /* batch handles: widest unit in words */
    int32_t frontier_build;  /* partial form, frontier engine: GUMAP_OPT_FRONTIER_BUILD value */
} gumap_tune_result;

/*
 * gumap_knn_autotune - pick the engine settings for this handle's graph by
 * timing gumap_knn_run (all vertices) on it: MS-BFS state budget (which
 * sets the source-block width), pull item width, heavy-vertex degree
 * multiplier, CTAs per SM (the CTA shape: registers per thread against
 * resident warps), staging of rows in shared memory and level direction
 * with its push threshold for the full form; engine and the frontier
 * engine's merge build for the partial form;
 * the widest unit (source-block width) for batch handles (no cache). The best settings are applied to the handle and, if cache_path is
 * not NULL, appended to that JSON-lines file under a key of the graph's
 * shape class (form, k, log2 n, log2 mean degree, hub ratio); a later
 * handle of the same class created while the environment variable
 * GUMAP_TUNE_CACHE names that file starts with them. If the cache already
 * holds the key, its settings are applied without timing. Synchronous;
 * allocates scratch outputs for the timing runs. (Library tuning, not a
 * step of the paper.) Errors: INVALID_ARG, OOM, CUDA.
 */
int gumap_knn_autotune(gumap_knn *h, const char *cache_path, gumap_tune_result *out);

/*
 * gumap_knn_get_stats - counters since the last reset. Synchronises the
 * device (it reads device-side level counters and CUDA events).
 */
int gumap_knn_get_stats(gumap_knn *h, gumap_knn_stats *out);
int gumap_knn_reset_stats(gumap_knn *h);

/* gumap_knn_destroy - free everything the handle owns (synchronises the device). NULL is allowed.
 * Device buffers go back to the library's pool (see gumap_pool_trim), so creating a handle of the
 * same shape again allocates nothing. */
int gumap_knn_destroy(gumap_knn *h);

/* gumap_pool_trim - return the pool's cached device buffers of `device` (-1: all devices) to CUDA.
 * The pool keeps at most GUMAP_POOL_BYTES (environment, default 8 GiB); beyond that, freed buffers
 * go straight back to CUDA. */
int gumap_pool_trim(int device);

/* Bytes the pool currently caches over all devices. */
int64_t gumap_pool_cached_bytes(void);

/*
 * gumap_knn_run_noalloc - kNN lists of every vertex (the same rows as
 * gumap_knn_run's out_idx / out_dist for sources == NULL) computed without
 * allocating anything. The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc where they need the lists, such as
 * code inside a framework that owns all device memory (a caching allocator
 * or a fixed budget) or a latency-bound loop that cannot afford cudaMalloc's
 * device synchronisation.
 *
 *   row_ptr, col_idx  device CSR (int32[n + 1], int32[nnz]) obeying the
 *                     gumap_knn_create rules; NOT validated here (validation
 *                     would need a synchronisation), so an invalid graph gives
 *                     undefined results.
 *   n, nnz, k, mode   as for gumap_knn_create (2 <= n; 1 <= k <= min(n-1, 256)).
 *   out_idx, out_dist device int32[n][k] / uint16[n][k], caller-owned.
 *   status_out        optional device int32[1]: receives GUMAP_OK or the
 *                     device status (GUMAP_ERR_TIMEOUT) when the work ends.
 *   stream            cudaStream_t; the call is asynchronous on it.
 *
 * All scratch comes from one 16 MiB file-scope device array inside the
 * library, which every GPU that loads the library holds until the process
 * exits. The call rejects graphs whose scratch would not fit (about
 * 3 * 16 + 4 bytes per vertex at the narrowest source block, i.e. n up to
 * roughly 320,000) with GUMAP_ERR_TOO_LARGE, and never calls cudaMalloc,
 * cudaFree or any allocating routine. The first call on a device looks up the
 * array's device address (make that first call before any stream capture).
 * Every call reuses the array and clears what must start at zero; calls whose
 * GPU work overlaps (other streams, other threads) race on it. Errors:
 * INVALID_ARG, TOO_LARGE, CUDA.
 */
int gumap_knn_run_noalloc(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int64_t nnz, int32_t k,
                          int mode, int32_t *out_idx, uint16_t *out_dist, int32_t *status_out, void *stream);

/* -------------------------------------------------- quality metrics -- */
/*
 * gumap_quality_np - neighbourhood preservation of a drawing X of the
 * handle's graph (Section 4.1.3): for each vertex v, N_G(v, r) is the set of
 * other vertices within r hops and N_D(v, r) the |N_G(v, r)| other vertices
 * closest to v in X; the metric is the sum over v of
 * |N_G cap N_D| / |N_G cup N_D| (the paper sets r = 2).
 *
 *   X          device float[n][dim], row-major: the drawing's coordinates.
 *   dim        1 .. 8.
 *   r          hop radius, >= 1.
 *   out_c      device int32[n] or NULL: |N_G(v, r)|.
 *   out_inter  device int32[n] or NULL: |N_G(v, r) cap N_D(v, r)|.
 *   out_sum    device double[1]: the sum over v (a vertex with an empty
 *              N_G(v, r) adds 1: two empty sets are identical).
 *
 * Closeness in X is the squared Euclidean distance in FP32 (each coordinate's
 * difference, its square and the running sum rounded to float in coordinate
 * order), ties broken by ascending vertex id; the counts are exact for that
 * order. Work grows as n^2 (every vertex ranks all others): n <= 2^20.
 * Asynchronous on `stream`. Errors: INVALID_ARG (batch handle, NULL pointer,
 * dim, r, n), OOM, CUDA.
 */
int gumap_quality_np(gumap_knn *h, const float *X, int32_t dim, int32_t r, int32_t *out_c, int32_t *out_inter,
                     double *out_sum, void *stream);

/*
 * gumap_quality_stress - aggregated stress of a drawing X of the handle's
 * graph (Section 4.1.3):
 *   1/(n^2 - n) * sum over ordered pairs i != j of ((d_ij - |X_i - X_j|) / d_ij)^2
 * with d_ij the hop distance (the all-pairs matrix of Algorithm 1, from the
 * bit-parallel BFS run to completion whatever the handle's form); a pair with
 * no connecting path adds 1, the limit of its term as d_ij grows without
 * bound (Section 3.2 gives such pairs an "infinite" distance).
 *
 *   X           device float[n][dim], row-major; dim 1 .. 8.
 *   out_rows    device double[n] or NULL: each row's sum over j.
 *   out_stress  device double[1]: the stress.
 *
 * Each term's difference d_ij - |X_i - X_j| is taken in FP64, its division
 * and square in FP32 (about 3e-7 relative), the sums in FP64. The handle keeps n^2
 * uint16 hop distances of scratch (n <= 65535). Asynchronous on `stream`.
 * Errors: INVALID_ARG (batch handle, NULL pointer, dim, n), OOM, CUDA;
 * device-side errors via gumap_knn_check().
 */
int gumap_quality_stress(gumap_knn *h, const float *X, int32_t dim, double *out_rows, double *out_stress,
                         void *stream);

/* -------------------------------------------------- spectral layout -- */
typedef struct {
    int32_t iterations;   /* Lanczos steps taken (over all restarts) */
    int32_t restarts;     /* restarts from the current Ritz vectors */
    double residual;      /* largest |M y - theta y| bound of the returned pairs */
    int32_t converged;    /* 1 when residual <= 1e-10 */
} gumap_spectral_info;

/*
 * gumap_spectral_layout - the spectral layout of the last run's kNN graph
 * G_k with its fuzzy-union weights W (the initial coordinates of the layout
 * stage, Algorithm 1's initialisation; Section 3.2, after Koren's spectral
 * graph drawing): the solutions x of L x = mu D x (L = D - W, D = diag(W 1))
 * for the `dim` smallest mu after the trivial mu = 0 (x constant), each
 * D-normalised (x^T D x = 1).
 *
 *   dim     1 .. 8 coordinates.
 *   out_X   device float[n][dim], row-major: column c is the c-th eigenvector;
 *           its sign makes the entry of largest magnitude (the first such
 *           vertex) positive; a vertex with no edge gets 0.
 *   out_mu  host double[dim] or NULL: the eigenvalues mu, ascending (NaN for
 *           a column the graph is too small to have).
 *   info    host, or NULL: iterations, restarts, residual bound.
 *
 * The handle's last gumap_knn_run must have built the union COO (union
 * weights). Eigenvectors of a repeated eigenvalue are any D-orthonormal basis
 * of its eigenspace; on a disconnected G_k only D^(1/2) 1 counts as trivial,
 * so the eigenvalue 0 of the other components comes first. One Lanczos run
 * per coordinate, with full reorthogonalisation in FP64 on the device (basis
 * of up to 400 vectors of n doubles, at most 4 GiB), each projecting out the
 * vectors found before and restarted from its Ritz vector until the residual
 * bound falls below 1e-10 (30 restarts at most). Synchronous on
 * `stream`. (Library extension: the paper's layout stage itself is out of
 * scope.) Errors: INVALID_ARG (no union COO, a union graph with no edge,
 * dim, NULL), OOM, CUDA.
 */
int gumap_spectral_layout(gumap_knn *h, int32_t dim, float *out_X, double *out_mu, gumap_spectral_info *info,
                          void *stream);

/* ------------------------------------------------------------ serving -- */
/*
 * A server computes the same rows as gumap_knn_run (kNN lists of every vertex
 * and their weights, Algorithm 1 / Algorithm 4, Section 2.1) for a stream of
 * independent graph requests. A native scheduler thread admits requests
 * while their device memory fits a fixed budget (one arena allocated at
 * creation, so nothing is allocated while serving), groups waiting small
 * graphs of equal k into one batched launch (gumap_batch_create's engine),
 * runs large graphs alone, and keeps several launches in flight on separate
 * streams (one of them reserved for small-graph batches, so long launches of
 * large graphs never hold every stream), so requests that arrive while others run are admitted as soon as
 * a stream and memory free up and their work overlaps on the device. Results
 * stay resident in the arena until released. All calls are thread-safe.
 */
typedef struct gumap_server gumap_server;

typedef struct {
    int32_t n_streams;          /* launches in flight at once (default 4)                      */
    int32_t max_batch_graphs;   /* graphs per batched launch (default 512)                     */
    int64_t max_batch_vertices; /* vertices per batched launch (default 4,000,000)             */
    int32_t max_queue;          /* waiting requests beyond which submit returns AGAIN (65536)  */
    int64_t staging_bytes;      /* pinned host staging for uploads (default 512 MiB)            */
    uint32_t flags;             /* GUMAP_WEIGHTS_* applied to every request (default union)    */
} gumap_server_opts;

typedef struct {
    int32_t status;             /* GUMAP_OK, GUMAP_PENDING or the request's error              */
    int32_t n, k;
    const int32_t *idx;         /* device int32[n][k], ids local to the request's graph        */
    const uint16_t *dist;       /* device uint16[n][k]                                          */
    const float *w;             /* device float[n][k]                                           */
    double t_submit, t_start, t_done; /* seconds on the server clock (gumap_server_clock)      */
    int32_t batch_graphs;       /* requests that shared this request's launch                   */
    int32_t engine;             /* GUMAP_ENGINE_* that ran it                                   */
} gumap_result;

typedef struct {
    int64_t submitted, completed, failed, released, launches, pending, running;
    int64_t arena_bytes, arena_used_bytes, arena_peak_bytes;
} gumap_server_stats;

/*
 * gumap_server_create - start a server on `device` whose requests may hold
 * at most hbm_budget_bytes of device memory (allocated once, here).
 * opts may be NULL (defaults). Errors: INVALID_ARG, OOM, CUDA.
 */
int gumap_server_create(gumap_server **s, int device, uint64_t hbm_budget_bytes, const gumap_server_opts *opts);

/*
 * gumap_serve_submit - queue one graph (host CSR obeying the gumap_knn_create
 * rules; validated and copied before returning, so the caller may free it).
 * k and mode as for gumap_knn_create. Non-blocking. Errors: INVALID_ARG,
 * INVALID_GRAPH, AGAIN (queue full: retry), TOO_LARGE (the request alone can
 * never fit the budget).
 */
int gumap_serve_submit(gumap_server *s, const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int64_t nnz,
                       int32_t k, int mode, uint64_t *req_id);

/* gumap_serve_poll - GUMAP_PENDING, GUMAP_OK (out filled) or an error; non-blocking. */
int gumap_serve_poll(gumap_server *s, uint64_t req_id, gumap_result *out);

/* gumap_serve_wait - like poll, but blocks up to timeout_s seconds (GUMAP_PENDING if still running). */
int gumap_serve_wait(gumap_server *s, uint64_t req_id, gumap_result *out, double timeout_s);

/* gumap_serve_read - copy a finished request's rows into caller buffers (device or host memory;
 * any may be NULL) on `stream`, asynchronously. Errors: UNKNOWN_REQUEST, PENDING, the request's error. */
int gumap_serve_read(gumap_server *s, uint64_t req_id, int32_t *idx, uint16_t *dist, float *w, void *stream);

/* gumap_serve_release - the request's result may be dropped; its memory returns to the budget once
 * every request of its launch is released. Errors: UNKNOWN_REQUEST. */
int gumap_serve_release(gumap_server *s, uint64_t req_id);

/* Seconds since the server started (the clock of gumap_result's timestamps). */
double gumap_server_clock(gumap_server *s);

int gumap_server_get_stats(gumap_server *s, gumap_server_stats *out);

/* gumap_server_destroy - stop the scheduler (finishing launched work), free everything. NULL allowed. */
int gumap_server_destroy(gumap_server *s);

/*
 * gumap_selftest_wait_timeout - check that a device-side wait of this library
 * gives up instead of hanging: launches the grid barrier of the multi-source
 * BFS with one CTA that never arrives and a limit of limit_s seconds
 * (1 ms .. 5 s), waits, and returns the status the waiting CTAs recorded:
 * GUMAP_ERR_TIMEOUT when the mechanism works. The context stays usable.
 * Synchronous. (Failure handling of the library, not a step of the paper.)
 */
int gumap_selftest_wait_timeout(int device, double limit_s);

/* Static string for a status code (never NULL). */
const char *gumap_status_string(int status);

/* Message of the calling thread's last failed call ("" if none). */
const char *gumap_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GUMAP_H */
