// Bit-parallel multi-source BFS (MS-BFS) with kNN extraction.
//
// One launch processes one block of up to 32*W sources. Each vertex row of
// the three bitsets holds one bit per source (vertex-major, W 32-bit words,
// W a multiple of 4 so a thread moves 128 bits with one uint4 access):
//   F[v]  frontier: sources that reached v at the previous level
//   N[v]  next:     sources that reach v at the current level
//   S[v]  seen:     sources that reached v at any level so far (F included)
// A level is the pull step  N[v] = (OR_{u in adj(v)} F[u]) & act & ~S[v],
// then S[v] |= N[v], which is one frontier expansion of the partial BFS of
// Algorithm 4 and of the BFS behind Algorithm 1's all-pairs distances, run
// for 32*W sources at once. The OR over neighbours stops as soon as every
// still-missing source bit is covered (the bottom-up early exit), and a
// vertex already reached by every active source costs no neighbour loads.
// Such a saturated item stays saturated (S only grows, act only shrinks):
// after writing its N word 0 in both buffers it is skipped for good (one
// state byte per item, read only once some item has saturated). In the full
// form each pull also counts the items that are saturated after it; when
// that is every item, the next level could reach nothing and is not run.
//
// Pull-only levels over a block of consecutive sources (every run over all
// vertices) use the seen sets alone: a source first reaches v at level d
// exactly when it had reached some neighbour of v by level d - 1 and not v,
// so S_d[v] = S_{d-1}[v] | ((OR_{u in adj(v)} S_{d-1}[u]) & act & ~S_{d-1}[v]).
// S_{d-1}, S_d and S_{d+1} rotate over the three buffers, a level reads one
// row stream and writes one (no frontier stream), and level d's new pairs,
// which the extraction needs, are S_d & ~S_{d-1}. A saturated item's state
// byte then counts the buffers already holding its final row (2, then 3),
// after which the item is skipped.
//
// Work of a level is the set of (vertex v, 128-bit group g) items. Items of
// vertices of ordinary degree are one thread each (the neighbour loop is
// short). Items of vertices whose degree is far above the mean (hubs of
// scale-free graphs) are one warp each, the lanes splitting the neighbour
// list and OR-reducing with shuffles, so no level waits on one thread
// walking a hub's adjacency. Both lists run in decreasing degree. In the
// staged build each CTA owns an interleaved slice of the ordinary vertices,
// whose neighbour ids it bulk-copies (cp.async.bulk, completion on an
// mbarrier) into shared memory once per launch. The slices also hold each
// hub's row cut into segments of at least 16 entries; the seen-set pull runs
// those segments like ordinary rows, every segment ORing what it finds into
// the hub's S_d row with atomics (exact, as the buffer held S_{d-3}, a
// subset of S_{d-1}), and then needs no warp-wide hub items.
//
// Level 1 of a block of consecutive sources (every run over all vertices)
// is a pull from the sorted rows that writes N and S in full (S_1 alone in
// the seen-set pull); for an
// explicit source list it is a push from the sources' rows into N only, and
// level 2 folds the level-1 frontier into S. Its kNN entries are the first
// k entries of each source's sorted CSR row. For later levels the
// extraction scans each word column of N (of S_d & ~S_{d-1} in the seen-set
// pull) in vertex order, transposes 32x32
// bit tiles with warp ballots, and appends to every incomplete source the
// vertices it reached at this level in ascending id until its list holds k
// entries: this is exactly the (distance, id) order, because levels are
// visited in increasing distance and vertices in increasing id. It runs in
// the same phase as the next level's pull, which only reads the same
// buffer. When all-pairs rows are requested every column is scanned and
// each newly reached (source, vertex) pair gets its distance. In the
// partial form (Algorithm 4, which stops a source once more than k
// vertices are visited) a source whose list is complete stops propagating:
// its bit leaves `act`. The full form keeps every source propagating until
// no source reaches a new vertex.
//
// All levels run inside one cooperative launch; phases are separated by a
// grid barrier whose waits are bounded in time (kWaitLimitNs).
#include "gumap_internal.cuh"

#include <algorithm>

namespace gumap {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int32_t* p) {
    return *reinterpret_cast<const volatile int32_t*>(p);
}

__device__ __forceinline__ unsigned ld_volatile_u32(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

// ---- bulk copy global -> shared (TMA engine), completion on an mbarrier

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the async (bulk-copy) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// dst, src 16-byte aligned, bytes a nonzero multiple of 16
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for phase `parity` of the barrier for at most limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned long long limit_ns) {
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}

// Grid-wide barrier for a cooperative launch. Thread 0 of each CTA arrives
// on a counter; the last arrival bumps the generation. Waiters poll the
// generation for at most limit_ns, then record a timeout and return false
// (every later barrier of that CTA is skipped by the caller).
__device__ bool grid_barrier(GridBarrier* bar, int32_t* status, unsigned long long limit_ns = kWaitLimitNs) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned nblocks = gridDim.x;
        unsigned gen0 = ld_acquire_u32(&bar->gen);
        __threadfence();
        unsigned prev = atomicAdd(&bar->count, 1u);
        if (prev == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            unsigned long long t0 = globaltimer_ns();
            while (ld_acquire_u32(&bar->gen) == gen0) {
                if (globaltimer_ns() - t0 > limit_ns) {
                    atomicExch(status, kStatusTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ uint4 or4(uint4 a, uint4 b) {
    return make_uint4(a.x | b.x, a.y | b.y, a.z | b.z, a.w | b.w);
}
__device__ __forceinline__ uint4 and4(uint4 a, uint4 b) {
    return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}
__device__ __forceinline__ uint4 andnot4(uint4 a, uint4 b) {  // a & ~b
    return make_uint4(a.x & ~b.x, a.y & ~b.y, a.z & ~b.z, a.w & ~b.w);
}
__device__ __forceinline__ bool nz4(uint4 a) { return (a.x | a.y | a.z | a.w) != 0u; }
// true when every bit of `todo` is present in `acc`
__device__ __forceinline__ bool covers4(uint4 acc, uint4 todo) { return !nz4(andnot4(todo, acc)); }

__device__ __forceinline__ uint4 ldcg4(const uint4* p) { return __ldcg(p); }

__device__ __forceinline__ uint4 warp_or4(uint4 a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a.x |= __shfl_xor_sync(kFull, a.x, o);
        a.y |= __shfl_xor_sync(kFull, a.y, o);
        a.z |= __shfl_xor_sync(kFull, a.z, o);
        a.w |= __shfl_xor_sync(kFull, a.w, o);
    }
    return a;
}

// ---------------------------------------------------------------- phases

// Zeroes the pull items' saturation states (see MsbfsArgs::sat).
__device__ __forceinline__ void clear_sat(const MsbfsArgs& a, long long tid, long long nthr) {
    if (!a.sat) return;
    const long long items = (long long)a.n * (a.W / (a.pull_width == 2 ? 2 : 4));
    uint4* s4 = reinterpret_cast<uint4*>(a.sat);
    for (long long i = tid; i < (items + 15) / 16; i += nthr) s4[i] = make_uint4(0u, 0u, 0u, 0u);
}

// Phase 0: clear S and N, prefill the block's output rows with padding,
// mark valid source bits in act/need.
__device__ void phase_init(const MsbfsArgs& a) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long words4 = (long long)a.n * (a.W >> 2);
    uint4* S4 = reinterpret_cast<uint4*>(a.S);
    uint4* N4 = reinterpret_cast<uint4*>(a.N);
    uint4* F4 = reinterpret_cast<uint4*>(a.F);
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    const bool clear_f = a.direction != 1;  // a push into F (level 2) needs it zero
    for (long long i = tid; i < words4; i += nthr) {
        S4[i] = z;
        N4[i] = z;
        if (clear_f) F4[i] = z;
    }
    if (a.inq)
        for (long long i = tid; i < a.n; i += nthr) a.inq[i] = 0;
    clear_sat(a, tid, nthr);
    for (long long i = tid; i < a.W; i += nthr) {
        long long lo = i * 32;
        uint32_t m;
        if (lo + 32 <= a.nb) m = kFull;
        else if (lo >= a.nb) m = 0u;
        else m = (1u << (a.nb - lo)) - 1u;
        a.act[i] = m;
        a.need[i] = m;
    }
    const long long slots = (long long)a.nb * a.k;
    for (long long i = tid; i < slots; i += nthr) {
        a.out_idx[i] = -1;
        a.out_dist[i] = kDistInf;
    }
    for (long long i = tid; i < a.nb; i += nthr) a.cnt[i] = 0;
    if (tid == 0) {  // the other per-launch counters were zeroed by the host
        a.ctr->n_need = a.nb;
        a.ctr->qvalid[0] = 1;  // F was cleared: the buffer level 2 writes holds no row
        a.ctr->u_edges[0] = (unsigned long long)__ldg(a.row_ptr + a.n) * (unsigned long long)(a.W >> 2);
    }
}

// Appends each lane's v (where want) to q with one atomic per warp. All 32
// lanes must call it together.
__device__ __forceinline__ void warp_append(bool want, int v, int32_t* q, int32_t* cnt) {
    const unsigned m = __ballot_sync(kFull, want);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (want) q[base + __popc(m & ((1u << lane) - 1u))] = v;
}

// Block-wide sum of a per-thread counter into a global one (one atomic per
// CTA). All threads of the CTA must call it.
__device__ __forceinline__ void block_add(unsigned long long x, unsigned long long* dst) {
    __shared__ unsigned long long s_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if (threadIdx.x == 0) s_acc = 0ull;
    __syncthreads();
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_acc, x);
    __syncthreads();
    if (threadIdx.x == 0 && s_acc) atomicAdd(dst, s_acc);
}

// Phases 0 and 1 in one pass for a block whose sources are the consecutive
// vertices src_lo .. src_lo + nb - 1 (every run over all vertices). Level 1
// is computed as a pull instead of pushed: N[v] = the block's sources
// adjacent to v, read off v's sorted row (one warp per vertex, 4096 source
// bits per round, each neighbour read once), and S[v] = v's own bit and
// N[v]; both rows are written in full, so nothing is cleared first and no
// atomics touch the bitsets. Each source's level-1 kNN entries (the first k of its row)
// and padding are written by one warp, the act/need masks one 32-source word
// per warp. The per-launch counters were zeroed by the host.
constexpr int kInitRound = 8;  // row entries per lane loaded together by the level-1 pull

template <bool SO>
__device__ void phase_init_identity(const MsbfsArgs& a) {
    __shared__ __align__(16) uint32_t s_chunk[8][128];  // per warp: 128 words = 4096 source bits
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const long long gwarp = gtid >> 5, nwarps = nthr >> 5;
    uint32_t* sc = s_chunk[(threadIdx.x >> 5) & 7];
    const int G4 = a.W >> 2;
    const int chunks = (a.W + 127) >> 7;
    uint4* N4 = reinterpret_cast<uint4*>(a.N);
    uint4* S4 = reinterpret_cast<uint4*>(a.S);
    uint4* F4 = reinterpret_cast<uint4*>(a.F);
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    const bool clear_f = a.direction != 1;  // a push into F (level 2) needs it zero
    const long long src_hi = (long long)a.src_lo + a.nb;
    int any = 0;
    unsigned long long fe = 0ull;
    clear_sat(a, gtid, nthr);
    for (long long v = gwarp; v < a.n; v += nwarps) {
        const int r0 = __ldg(a.row_ptr + v), r1 = __ldg(a.row_ptr + v + 1);
        int lo = r0, hi = r1;  // first neighbour >= src_lo (every one when the block starts at vertex 0)
        while (a.src_lo > 0 && lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(a.col + mid) < a.src_lo) lo = mid + 1;
            else hi = mid;
        }
        int e = lo;
        const long long j = v - a.src_lo;  // v's bit in the block, if v is one of its sources
        for (int c = 0; c < chunks; ++c) {
            reinterpret_cast<uint4*>(sc)[lane] = z;
            __syncwarp();
            const long long base = (long long)a.src_lo + 4096ll * c;
            const long long top = base + 4096 < src_hi ? base + 4096 : src_hi;
            // the neighbours in [base, top) are the next entries of the sorted row;
            // kInitRound of them per lane are loaded at once
            while (true) {
                long long u[kInitRound];
#pragma unroll
                for (int j = 0; j < kInitRound; ++j) {
                    const int idx = e + 32 * j + lane;
                    u[j] = idx < r1 ? (long long)__ldg(a.col + idx) : src_hi;
                }
                int taken = 0;
#pragma unroll
                for (int j = 0; j < kInitRound; ++j) {
                    const bool in = u[j] < top;
                    if (in) atomicOr(&sc[(u[j] - base) >> 5], 1u << ((u[j] - base) & 31));
                    taken += __popc(__ballot_sync(kFull, in));
                }
                e += taken;  // the row is sorted: the entries below top are a prefix
                if (taken < 32 * kInitRound) break;
            }
            __syncwarp();
            const int g = c * 32 + lane;
            if (g < G4) {
                const uint4 nbits = reinterpret_cast<const uint4*>(sc)[lane];
                const size_t off = (size_t)v * G4 + g;
                if (!SO) N4[off] = nbits;
                uint4 sbits = z;
                if (j >= 0 && j < a.nb && (j >> 7) == g) {
                    const uint32_t bit = 1u << (j & 31);
                    const int wi = (int)((j >> 5) & 3);
                    sbits.x = wi == 0 ? bit : 0u;
                    sbits.y = wi == 1 ? bit : 0u;
                    sbits.z = wi == 2 ? bit : 0u;
                    sbits.w = wi == 3 ? bit : 0u;
                }
                if (SO) {
                    N4[off] = or4(sbits, nbits);  // S_1 in buffer 1 % 3 (N)
                } else {
                    S4[off] = or4(sbits, nbits);  // S holds levels 0 and 1: level 2 needs no fold
                    if (clear_f) F4[off] = z;
                }
                if (nz4(nbits)) {
                    any = 1;
                    fe += (unsigned long long)(r1 - r0);
                }
            }
            __syncwarp();
        }
        if (a.inq && lane == 0) a.inq[v] = 0;
    }
    // seen-set pull with hub segments: the hubs' rows of the buffers of S_2
    // and S_3, which segments OR into, start empty
    if (SO && a.hub_segments) {
        const long long items = (long long)a.n_heavy * G4;
        for (long long t = gtid; t < items; t += nthr) {
            const long long h = t / G4;
            const size_t off = (size_t)__ldg(a.heavy + h) * G4 + (size_t)(t - h * G4);
            F4[off] = z;
            S4[off] = z;
        }
    }
    // level-1 kNN entries of each source and the padding after them
    for (long long jj = gwarp; jj < a.nb; jj += nwarps) {
        const int s = a.src_lo + (int)jj;
        const int e0 = __ldg(a.row_ptr + s), e1 = __ldg(a.row_ptr + s + 1);
        const int take = e1 - e0 < a.k ? e1 - e0 : a.k;
        int32_t* oi = a.out_idx + (size_t)jj * a.k;
        uint16_t* od = a.out_dist + (size_t)jj * a.k;
        for (int t = lane; t < a.k; t += 32) {
            oi[t] = t < take ? __ldg(a.col + e0 + t) : -1;
            od[t] = t < take ? (uint16_t)1 : kDistInf;
        }
        if (lane == 0) a.cnt[jj] = take;
        if (a.apsp) {  // distances 0 and 1 of the all-pairs row
            uint16_t* row = a.apsp + (size_t)jj * a.apsp_ld;
            if (lane == 0) row[s] = 0;
            for (int e = e0 + lane; e < e1; e += 32) row[__ldg(a.col + e)] = 1;
        }
    }
    // act / need, one word of 32 sources per warp: a source whose row holds
    // k entries has its list; one with an empty row is finished and silent
    for (long long w = gwarp; w < a.W; w += nwarps) {
        const long long jj = w * 32 + lane;
        const bool valid = jj < a.nb;
        const int d = valid ? __ldg(a.row_ptr + a.src_lo + jj + 1) - __ldg(a.row_ptr + a.src_lo + jj) : 0;
        const unsigned vm = __ballot_sync(kFull, valid);
        const unsigned dm = __ballot_sync(kFull, valid && (d >= a.k || d == 0));
        const unsigned zm = __ballot_sync(kFull, valid && d == 0);
        if (lane == 0) {
            a.need[w] = vm & ~dm;
            a.act[w] = vm & ~(a.partial ? dm : zm);
            if (vm & ~dm) atomicAdd(&a.ctr->n_need, __popc(vm & ~dm));
        }
    }
    if (gtid == 0) {
        a.ctr->qvalid[0] = 1;
        a.ctr->u_edges[0] = (unsigned long long)__ldg(a.row_ptr + a.n) * (unsigned long long)(a.W >> 2);
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(&a.ctr->lvl_any[1], 1u);
    if (a.direction == 0) block_add(fe, &a.ctr->f_edges[1]);
}

// Phase 1: seed S with the sources (level 0), push level 1 into N, and take
// the level-1 kNN entries straight from each source's sorted CSR row.
__device__ void phase_seed(const MsbfsArgs& a) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    for (long long j = tid; j < a.nb; j += nthr) {
        const int s = a.src[j];
        if (s >= 0 && s < a.n) atomicOr(&a.S[(size_t)s * a.W + (j >> 5)], 1u << (j & 31));
    }
    const int lane = threadIdx.x & 31;
    const long long warp = tid >> 5;
    const long long nwarps = nthr >> 5;
    int any = 0;
    unsigned long long fe = 0ull;  // edges leaving the level-1 frontier (for the direction choice)
    for (long long j = warp; j < a.nb; j += nwarps) {
        const int s = a.src[j];
        const bool ok = s >= 0 && s < a.n;  // an invalid source is an empty row
        if (!ok && lane == 0) atomicExch(&a.ctr->status, kStatusBadSource);
        const int e0 = ok ? __ldg(a.row_ptr + s) : 0, e1 = ok ? __ldg(a.row_ptr + s + 1) : 0;
        const int deg = e1 - e0;
        const uint32_t bit = 1u << (j & 31);
        uint32_t* Ncol = a.N + (j >> 5);
        for (int e = e0 + lane; e < e1; e += 32) {
            const int u = __ldg(a.col + e);
            atomicOr(Ncol + (size_t)u * a.W, bit);
            fe += (unsigned long long)(__ldg(a.row_ptr + u + 1) - __ldg(a.row_ptr + u));
        }
        const int take = deg < a.k ? deg : a.k;
        int32_t* oi = a.out_idx + (size_t)j * a.k;
        uint16_t* od = a.out_dist + (size_t)j * a.k;
        for (int t = lane; t < take; t += 32) {
            oi[t] = __ldg(a.col + e0 + t);
            od[t] = 1;
        }
        if (a.apsp && ok) {  // distances 0 and 1 of the all-pairs row
            uint16_t* row = a.apsp + (size_t)j * a.apsp_ld;
            if (lane == 0) row[s] = 0;
            for (int e = e0 + lane; e < e1; e += 32) row[__ldg(a.col + e)] = 1;
        }
        if (lane == 0) {
            a.cnt[j] = take;
            if (deg > 0) any = 1;
            if (take >= a.k || deg == 0) {
                atomicAnd(&a.need[j >> 5], ~bit);
                if (a.partial || deg == 0) atomicAnd(&a.act[j >> 5], ~bit);
                atomicSub(&a.ctr->n_need, 1);
            }
        }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(&a.ctr->lvl_any[1], 1u);
    block_add(fe, &a.ctr->f_edges[1]);
}

// Vector helpers of the pull for its two item widths: a thread owns either a
// 128-bit group (uint4, four words) or a 64-bit group (uint2, two words) of
// a vertex row.
template <int GW> struct PullVec;
template <> struct PullVec<4> { using T = uint4; };
template <> struct PullVec<2> { using T = uint2; };

__device__ __forceinline__ uint4 vzero(uint4) { return make_uint4(0u, 0u, 0u, 0u); }
__device__ __forceinline__ uint2 vzero(uint2) { return make_uint2(0u, 0u); }
__device__ __forceinline__ uint4 vor(uint4 a, uint4 b) { return or4(a, b); }
__device__ __forceinline__ uint2 vor(uint2 a, uint2 b) { return make_uint2(a.x | b.x, a.y | b.y); }
__device__ __forceinline__ uint4 vand(uint4 a, uint4 b) { return and4(a, b); }
__device__ __forceinline__ uint2 vand(uint2 a, uint2 b) { return make_uint2(a.x & b.x, a.y & b.y); }
__device__ __forceinline__ uint4 vandnot(uint4 a, uint4 b) { return andnot4(a, b); }
__device__ __forceinline__ uint2 vandnot(uint2 a, uint2 b) { return make_uint2(a.x & ~b.x, a.y & ~b.y); }
__device__ __forceinline__ bool vnz(uint4 a) { return nz4(a); }
__device__ __forceinline__ bool vnz(uint2 a) { return (a.x | a.y) != 0u; }
__device__ __forceinline__ uint4 vld(const uint4* p) { return __ldcg(p); }
__device__ __forceinline__ uint2 vld(const uint2* p) { return __ldcg(p); }
__device__ __forceinline__ uint4 vwarp_or(uint4 a) { return warp_or4(a); }
__device__ __forceinline__ uint2 vwarp_or(uint2 a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a.x |= __shfl_xor_sync(kFull, a.x, o);
        a.y |= __shfl_xor_sync(kFull, a.y, o);
    }
    return a;
}
template <typename T>
__device__ __forceinline__ bool vcovers(T acc, T todo) { return !vnz(vandnot(todo, acc)); }

// A CTA's view of its staged slice (see MsbfsArgs): mode 0 = not staged
// (light items spread over the grid, rows from the global CSR); 1 = the
// slice's (vertex, offset) pairs and neighbour ids in shared memory; 2 = the
// same slice read from global memory (the bulk copy did not complete).
struct StageView {
    const int2* meta;     // pairs of positions p0 .. p0 + P
    const int32_t* col;   // neighbour ids; an offset o of meta is col[o - cbase]
    int32_t P;
    int32_t cbase;
    int32_t mode;
};

// One light (vertex v, group g) item of the pull: the OR of the neighbours'
// frontier groups over the ids col[e0, e1), stopping once every missing
// source is covered. SLICE: col is a staged slice (plain loads; shared
// memory, or global memory when the copy failed), else the global CSR (read
// through the read-only path). NB neighbour loads are in flight at once.
template <int GW, int NB, bool SLICE>
__device__ __forceinline__ void pull_light_item(const typename PullVec<GW>::T* __restrict__ FV,
                                                typename PullVec<GW>::T* __restrict__ NV,
                                                typename PullVec<GW>::T* __restrict__ SV,
                                                const typename PullVec<GW>::T* __restrict__ actV, int G, int g, int v,
                                                const int32_t* __restrict__ col, int e0, int e1, bool fold,
                                                uint8_t* __restrict__ sat, bool use_sat, unsigned long long& fe,
                                                unsigned long long& ue, int& any, unsigned& nsat, int& newsat) {
    using VT = typename PullVec<GW>::T;
    const VT zero = vzero(VT{});
    const size_t off = (size_t)v * G + g;
    if (use_sat) {  // a saturated item: zero the N buffer once more, then skip it for good
        const uint8_t st = sat[off];
        if (st == 2) {
            ++nsat;
            return;
        }
        if (st == 1) {
            NV[off] = zero;
            sat[off] = 2;
            ++nsat;
            return;
        }
    }
    const VT s0 = vld(SV + off);
    const VT seen = fold ? vor(s0, vld(FV + off)) : s0;
    const VT todo = vandnot(vld(actV + g), seen);
    VT acc = zero;
    if (vnz(todo)) {
        const VT* fg = FV + g;
        for (int e = e0; e < e1; e += NB) {
            int u[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) u[q] = (e + q < e1) ? (SLICE ? col[e + q] : __ldg(col + e + q)) : -1;
            VT f[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) f[q] = u[q] >= 0 ? vld(fg + (size_t)u[q] * G) : zero;
#pragma unroll
            for (int q = 0; q < NB; ++q) acc = vor(acc, f[q]);
            if (vcovers(acc, todo)) break;
        }
        acc = vand(acc, todo);
        const unsigned long long dv = (unsigned long long)(e1 - e0);
        if (vnz(acc)) fe += dv;
        if (vnz(vandnot(todo, acc))) ue += dv;
    }
    NV[off] = acc;
    const VT s1 = vor(seen, acc);
    if (vnz(vandnot(s1, s0))) SV[off] = s1;
    any |= vnz(acc) ? 1 : 0;
    if (sat && !vnz(todo)) {
        sat[off] = 1;
        newsat = 1;
    }
    if (!vnz(vandnot(todo, acc))) ++nsat;  // every active source has now reached v
}

// A light item of the seen-set pull (MsbfsArgs::seen_only): PV holds
// S_{d-1}, CV receives S_d. The state byte counts the buffers that already
// hold a saturated item's final row: 2 after the level that found it
// saturated (S_{d-1} and S_d), 3 one level later, and from then on the item
// is skipped.
template <int GW, int NB, bool SLICE>
__device__ __forceinline__ void pull_seen_item(const typename PullVec<GW>::T* __restrict__ PV,
                                               typename PullVec<GW>::T* __restrict__ CV,
                                               const typename PullVec<GW>::T* __restrict__ actV, int G, int g, int v,
                                               const int32_t* __restrict__ col, int e0, int e1,
                                               uint8_t* __restrict__ sat, bool use_sat, unsigned long long& fe,
                                               unsigned long long& ue, int& any, unsigned& nsat, int& newsat) {
    using VT = typename PullVec<GW>::T;
    const VT zero = vzero(VT{});
    const size_t off = (size_t)v * G + g;
    const unsigned st = use_sat ? sat[off] : 0u;
    if (st == 3) {
        ++nsat;
        return;
    }
    const VT own = vld(PV + off);
    const VT todo = vandnot(vld(actV + g), own);
    if (!vnz(todo)) {  // saturated: carry the row into level d's buffer
        CV[off] = own;
        if (sat) {
            sat[off] = st == 2 ? 3 : 2;
            newsat = 1;
        }
        ++nsat;
        return;
    }
    VT acc = zero;
    const VT* fg = PV + g;
    for (int e = e0; e < e1; e += NB) {
        int u[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) u[q] = (e + q < e1) ? (SLICE ? col[e + q] : __ldg(col + e + q)) : -1;
        VT f[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) f[q] = u[q] >= 0 ? vld(fg + (size_t)u[q] * G) : zero;
#pragma unroll
        for (int q = 0; q < NB; ++q) acc = vor(acc, f[q]);
        if (vcovers(acc, todo)) break;
    }
    acc = vand(acc, todo);
    const unsigned long long dv = (unsigned long long)(e1 - e0);
    if (vnz(acc)) fe += dv;
    if (vnz(vandnot(todo, acc))) ue += dv;
    else ++nsat;  // every active source has now reached v
    CV[off] = vor(own, acc);
    any |= vnz(acc) ? 1 : 0;
}

__device__ __forceinline__ void vatomic_or(uint32_t* p, uint4 v) {
    if (v.x) atomicOr(p + 0, v.x);
    if (v.y) atomicOr(p + 1, v.y);
    if (v.z) atomicOr(p + 2, v.z);
    if (v.w) atomicOr(p + 3, v.w);
}
__device__ __forceinline__ void vatomic_or(uint32_t* p, uint2 v) {
    if (v.x) atomicOr(p + 0, v.x);
    if (v.y) atomicOr(p + 1, v.y);
}

// One segment (row entries col[e0, e1), staged) of a hub's item (v, g) in
// the seen-set pull. The segments of an item run in any order on any CTAs:
// each ORs what it finds into S_d[v][g] with atomics, segment 0 also ORs
// S_{d-1}[v][g]. The buffer of S_d held S_{d-3} (or zero, at levels 2 and
// 3), a subset of S_{d-1}, so the result is exactly S_{d-1} | found, with no
// initialisation and no finishing step. A saturated item's row is stored by
// every segment that sees it (the same value); its state byte is advanced by
// segment 0 alone, so a segment that reads the byte after segment 0 advanced
// it in the same level only stores the row again or skips, never advancing
// it twice (which would mark a buffer final that was not written).
// Segment 0 also counts the item.
template <int GW, int NB>
__device__ __forceinline__ void pull_seen_segment(const typename PullVec<GW>::T* __restrict__ PV,
                                                  typename PullVec<GW>::T* __restrict__ CV,
                                                  const typename PullVec<GW>::T* __restrict__ actV, int G, int g,
                                                  int v, bool first, const int32_t* __restrict__ col, int e0, int e1,
                                                  uint8_t* __restrict__ sat, bool use_sat, int& any, unsigned& nsat,
                                                  int& newsat) {
    using VT = typename PullVec<GW>::T;
    const VT zero = vzero(VT{});
    const size_t off = (size_t)v * G + g;
    const unsigned st = use_sat ? sat[off] : 0u;
    if (st == 3) {
        if (first) ++nsat;
        return;
    }
    const VT own = vld(PV + off);
    const VT todo = vandnot(vld(actV + g), own);
    if (!vnz(todo)) {
        CV[off] = own;
        if (sat && first) {
            sat[off] = st == 2 ? 3 : 2;
            newsat = 1;
        }
        if (first) ++nsat;
        return;
    }
    VT acc = zero;
    const VT* fg = PV + g;
    for (int e = e0; e < e1; e += NB) {
        int u[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) u[q] = (e + q < e1) ? col[e + q] : -1;
        VT f[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) f[q] = u[q] >= 0 ? vld(fg + (size_t)u[q] * G) : zero;
#pragma unroll
        for (int q = 0; q < NB; ++q) acc = vor(acc, f[q]);
        if (vcovers(acc, todo)) break;
    }
    acc = vand(acc, todo);
    any |= vnz(acc) ? 1 : 0;
    vatomic_or(reinterpret_cast<uint32_t*>(CV + off), first ? vor(own, acc) : acc);
}

// Pull step of level d (see file comment), with items of GW words. At level
// 2 the frontier F (level 1) is not yet in S: it is ORed in here. Also
// measures, for the choice of the next level's direction, the edges of the
// new frontier (sum of deg(v) over nonzero (v, group) items: what a push
// would touch) and of the items still unvisited (what the next pull would
// touch at most).
// SO (seen-set pull): Fc holds S_{d-1}, Nc receives S_d, a.S is not used.
template <int GW, int NB, bool STAGED, bool SO>
__device__ void phase_pull(const MsbfsArgs& a, const uint32_t* __restrict__ Fc, uint32_t* __restrict__ Nc,
                           int slot, int d, const StageView& sv) {
    using VT = typename PullVec<GW>::T;
    unsigned long long fe = 0ull, ue = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctr->qvalid[d % 4] = 0;  // a pull builds no queue
    const int G = a.W / GW;
    const int lane = threadIdx.x & 31;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const VT* FV = reinterpret_cast<const VT*>(Fc);
    VT* NV = reinterpret_cast<VT*>(Nc);
    VT* SV = reinterpret_cast<VT*>(a.S);
    const bool fold = d == 2 && !a.identity;  // the level-1 frontier is not yet in S
    const VT* actV = reinterpret_cast<const VT*>(a.act);
    const VT zero = vzero(VT{});
    int any = 0;
    unsigned nsat = 0;
    // A light item's saturation state is read only once some item has
    // saturated: before that every state byte is 0 and the loads are wasted.
    const bool use_sat = a.sat && ld_volatile_u32(&a.ctr->sat_seen) != 0u;
    int newsat = 0;

    // heavy vertices: one warp per (v, g), lanes split the neighbour list
    const long long heavy_items = (SO && STAGED && a.hub_segments) ? 0 : (long long)a.n_heavy * G;
    for (long long it = gtid >> 5; it < heavy_items; it += nthr >> 5) {
        const int h = (int)(it / G);
        const int g = (int)(it - (long long)h * G);
        const int v = __ldg(a.heavy + h);
        const size_t off = (size_t)v * G + g;
        if constexpr (SO) {  // seen-set pull: FV holds S_{d-1}, NV receives S_d
            const unsigned st = use_sat ? a.sat[off] : 0u;  // uniform over the warp
            if (st == 3) {
                if (lane == 0) ++nsat;
                continue;
            }
            const VT own = vld(FV + off);
            const VT todo = vandnot(vld(actV + g), own);
            if (!vnz(todo)) {
                if (lane == 0) {
                    NV[off] = own;
                    if (a.sat) {
                        a.sat[off] = st == 2 ? 3 : 2;
                        newsat = 1;
                    }
                    ++nsat;
                }
                continue;
            }
            VT acc = zero;
            const int e0 = __ldg(a.row_ptr + v), e1 = __ldg(a.row_ptr + v + 1);
            for (int base = e0; base < e1; base += 64) {
                const int ea = base + lane, eb = base + 32 + lane;
                const int ua = ea < e1 ? __ldg(a.col + ea) : -1;
                const int ub = eb < e1 ? __ldg(a.col + eb) : -1;
                if (ua >= 0) acc = vor(acc, vld(FV + (size_t)ua * G + g));
                if (ub >= 0) acc = vor(acc, vld(FV + (size_t)ub * G + g));
                acc = vwarp_or(acc);
                if (vcovers(acc, todo)) break;
            }
            acc = vand(acc, todo);
            if (lane == 0) {
                const unsigned long long dv = (unsigned long long)(e1 - e0);
                if (vnz(acc)) fe += dv;
                if (vnz(vandnot(todo, acc))) ue += dv;
                else ++nsat;
                NV[off] = vor(own, acc);
                any |= vnz(acc) ? 1 : 0;
            }
            continue;
        }
        if (a.sat) {  // the whole warp reads the same state: uniform branches
            const uint8_t st = a.sat[off];
            if (st == 2) {
                if (lane == 0) ++nsat;
                continue;
            }
            if (st == 1) {
                if (lane == 0) {
                    NV[off] = zero;
                    a.sat[off] = 2;
                    ++nsat;
                }
                continue;
            }
        }
        const VT s0 = vld(SV + off);
        const VT seen = fold ? vor(s0, vld(FV + off)) : s0;
        const VT todo = vandnot(vld(actV + g), seen);
        VT acc = zero;
        if (vnz(todo)) {
            const int e0 = __ldg(a.row_ptr + v), e1 = __ldg(a.row_ptr + v + 1);
            for (int base = e0; base < e1; base += 64) {
                const int ea = base + lane, eb = base + 32 + lane;
                const int ua = ea < e1 ? __ldg(a.col + ea) : -1;
                const int ub = eb < e1 ? __ldg(a.col + eb) : -1;
                if (ua >= 0) acc = vor(acc, vld(FV + (size_t)ua * G + g));
                if (ub >= 0) acc = vor(acc, vld(FV + (size_t)ub * G + g));
                acc = vwarp_or(acc);
                if (vcovers(acc, todo)) break;
            }
            acc = vand(acc, todo);
            if (lane == 0) {
                const unsigned long long dv = (unsigned long long)(e1 - e0);
                if (vnz(acc)) fe += dv;
                if (vnz(vandnot(todo, acc))) ue += dv;
            }
        }
        if (lane == 0) {
            NV[off] = acc;
            const VT s1 = vor(seen, acc);
            if (vnz(vandnot(s1, s0))) SV[off] = s1;
            any |= vnz(acc) ? 1 : 0;
            if (a.sat && !vnz(todo)) {
                a.sat[off] = 1;
                newsat = 1;
            }
            if (!vnz(vandnot(todo, acc))) ++nsat;
        }
    }

    // light vertices: one thread per (v, g), eight neighbour loads in flight.
    // An item index t = position * G + g advances by the stride as a
    // (position, group) pair: no division per item.
    if (!STAGED) {  // rows from the global CSR, items over the whole grid
        const int step_li = (int)(nthr / G), step_g = (int)(nthr - (long long)step_li * G);
        int li = (int)(gtid / G), g = (int)(gtid - (long long)li * G);
        while (li < a.n_light) {
            const int v = __ldg(a.light + li);
            if constexpr (SO)
                pull_seen_item<GW, NB, false>(FV, NV, actV, G, g, v, a.col, __ldg(a.row_ptr + v),
                                              __ldg(a.row_ptr + v + 1), a.sat, use_sat, fe, ue, any, nsat, newsat);
            else
                pull_light_item<GW, NB, false>(FV, NV, SV, actV, G, g, v, a.col, __ldg(a.row_ptr + v),
                                               __ldg(a.row_ptr + v + 1), fold, a.sat, use_sat, fe, ue, any, nsat,
                                               newsat);
            li += step_li;
            g += step_g;
            if (g >= G) {
                g -= G;
                ++li;
            }
        }
    } else {  // this CTA's slice of positions, rows from shared memory (mode 1) or global (mode 2)
        const int B = (int)blockDim.x;
        const int step_pi = B / G, step_g = B - step_pi * G;
        int pi = (int)threadIdx.x / G, g = (int)threadIdx.x - pi * G;
        while (pi < sv.P) {
            const int2 m0 = sv.meta[pi], m1 = sv.meta[pi + 1];
            if (m0.x < 0) {  // a hub segment: the seen-set pull runs it, the frontier scheme's heavy items cover it
                if constexpr (SO) {
                    const int hs = ~m0.x;
                    pull_seen_segment<GW, NB>(FV, NV, actV, G, g, __ldg(a.heavy + hs / kHubSegMax),
                                              hs % kHubSegMax == 0, sv.col, m0.y - sv.cbase, m1.y - sv.cbase, a.sat,
                                              use_sat, any, nsat, newsat);
                }
            } else if constexpr (SO) {
                pull_seen_item<GW, NB, true>(FV, NV, actV, G, g, m0.x, sv.col, m0.y - sv.cbase, m1.y - sv.cbase,
                                             a.sat, use_sat, fe, ue, any, nsat, newsat);
            } else {
                pull_light_item<GW, NB, true>(FV, NV, SV, actV, G, g, m0.x, sv.col, m0.y - sv.cbase, m1.y - sv.cbase,
                                              fold, a.sat, use_sat, fe, ue, any, nsat, newsat);
            }
            pi += step_pi;
            g += step_g;
            if (g >= G) {
                g -= G;
                ++pi;
            }
        }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(&a.ctr->lvl_any[slot], 1u);
    if (!a.partial) block_add(nsat, &a.ctr->sat_items[d % 4]);
    if (__syncthreads_or(newsat) && threadIdx.x == 0 && !use_sat) atomicOr(&a.ctr->sat_seen, 1u);
    if (a.direction == 0) {  // the statistics only feed the automatic choice
        block_add(fe, &a.ctr->f_edges[d % 4]);
        block_add(ue, &a.ctr->u_edges[d % 4]);
    }
}

// Preparation of a push level d: (a) if level d-1 was a pull, list the
// vertices of its frontier (rows of F with a nonzero group) into queue
// d-1; (b) clear the buffer level d writes (it holds level d-2): only the
// rows of queue d-2 when that queue exists, else all of it.
__device__ void phase_push_prep(const MsbfsArgs& a, const uint32_t* __restrict__ Fc, uint32_t* __restrict__ Nc,
                                int d) {
    const int G = a.W >> 2;
    const int lane = threadIdx.x & 31;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const uint4* F4 = reinterpret_cast<const uint4*>(Fc);
    uint4* N4 = reinterpret_cast<uint4*>(Nc);
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    if (!ld_volatile_i32(&a.ctr->qvalid[(d - 1) % 4])) {
        int32_t* q = a.queue + (size_t)((d - 1) % 4) * a.n;
        for (long long t0 = gtid & ~31ll; t0 < a.n; t0 += nthr) {
            const int v = (int)(t0 + lane);
            bool nzrow = false;
            if (v < a.n) {
                const uint4* row = F4 + (size_t)v * G;
                for (int g = 0; g < G && !nzrow; ++g) nzrow = nz4(ldcg4(row + g));
                if (nzrow) a.inq[v] = d - 1;
            }
            warp_append(nzrow, v, q, &a.ctr->qcnt[(d - 1) % 4]);
        }
    }
    if (ld_volatile_i32(&a.ctr->qvalid[(d - 2) % 4])) {
        const int32_t* q = a.queue + (size_t)((d - 2) % 4) * a.n;
        const long long items = (long long)ld_volatile_i32(&a.ctr->qcnt[(d - 2) % 4]) * G;
        for (long long t = gtid; t < items; t += nthr) {
            const long long i = t / G;
            N4[(size_t)__ldcg(q + i) * G + (t - i * G)] = z;
        }
    } else {
        const long long words4 = (long long)a.n * G;
        for (long long t = gtid; t < words4; t += nthr) N4[t] = z;
    }
    // the queue-valid flags change only in phase_push, after the barrier that
    // ends this phase: every CTA must read the same values here
}

// Push step of level d: one warp per (frontier vertex u, group g), lanes over
// u's neighbours v, each ORing F[u][g] & act & ~S[v] into N[v][g] and S[v][g];
// v joins queue d the first time it gains a bit. Bits that another warp
// adds to S[v] during the level are already in N[v], so reading S[v] while
// it grows loses nothing. At level 2 of an explicit source list the
// level-1 frontier is not yet in S:
// each queue item folds F[u][g] into S[u][g] (atomically, as other warps
// may be adding to the same row) and the mask also excludes F[v].
__device__ void phase_push(const MsbfsArgs& a, const uint32_t* __restrict__ Fc, uint32_t* __restrict__ Nc, int d) {
    const int G = a.W >> 2;
    const int lane = threadIdx.x & 31;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const uint4* F4 = reinterpret_cast<const uint4*>(Fc);
    const uint4* S4 = reinterpret_cast<const uint4*>(a.S);
    const uint4* act4 = reinterpret_cast<const uint4*>(a.act);
    const bool fold = d == 2 && !a.identity;  // the level-1 frontier is not yet in S
    const int32_t* qin = a.queue + (size_t)((d - 1) % 4) * a.n;
    int32_t* qout = a.queue + (size_t)(d % 4) * a.n;
    const long long items = (long long)ld_volatile_i32(&a.ctr->qcnt[(d - 1) % 4]) * G;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctr->qvalid[(d - 1) % 4] = 1;  // compacted by the prep phase if it was missing
        a.ctr->qvalid[d % 4] = 1;        // built by this phase
    }
    int any = 0;
    unsigned long long fe = 0ull;
    for (long long it = gwarp; it < items; it += nwarps) {
        const long long i = it / G;
        const int g = (int)(it - i * G);
        const int u = __ldcg(qin + i);
        const size_t uo = (size_t)u * G + g;
        const uint4 f = ldcg4(F4 + uo);
        if (!nz4(f)) continue;
        if (fold && lane == 0) {
            uint32_t* su = a.S + uo * 4;
            if (f.x) atomicOr(su + 0, f.x);
            if (f.y) atomicOr(su + 1, f.y);
            if (f.z) atomicOr(su + 2, f.z);
            if (f.w) atomicOr(su + 3, f.w);
        }
        const uint4 fa = and4(f, ldcg4(act4 + g));
        if (!nz4(fa)) continue;
        const int e0 = __ldg(a.row_ptr + u), e1 = __ldg(a.row_ptr + u + 1);
        for (int base = e0; base < e1; base += 32) {
            const int e = base + lane;
            const int v = e < e1 ? __ldg(a.col + e) : 0;
            bool want = false;
            if (e < e1) {
                const size_t vo = (size_t)v * G + g;
                const uint4 sv = ldcg4(S4 + vo);
                const uint4 m = andnot4(fa, fold ? or4(sv, ldcg4(F4 + vo)) : sv);
                if (nz4(m)) {
                    uint32_t* nw = Nc + vo * 4;
                    uint32_t* sw = a.S + vo * 4;
                    bool fresh = true;
                    if (m.x) fresh &= atomicOr(nw + 0, m.x) == 0u;
                    if (m.y) fresh &= atomicOr(nw + 1, m.y) == 0u;
                    if (m.z) fresh &= atomicOr(nw + 2, m.z) == 0u;
                    if (m.w) fresh &= atomicOr(nw + 3, m.w) == 0u;
                    if (m.x) atomicOr(sw + 0, m.x);
                    if (m.y) atomicOr(sw + 1, m.y);
                    if (m.z) atomicOr(sw + 2, m.z);
                    if (m.w) atomicOr(sw + 3, m.w);
                    if (fresh) fe += (unsigned long long)(__ldg(a.row_ptr + v + 1) - __ldg(a.row_ptr + v));
                    any = 1;
                    want = ld_volatile_i32(a.inq + v) != d && atomicExch(a.inq + v, d) != d;
                }
            }
            warp_append(want, v, qout, &a.ctr->qcnt[d % 4]);
        }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(&a.ctr->lvl_any[d % 3], 1u);
    block_add(fe, &a.ctr->f_edges[d % 4]);
}

// Extraction of level d: one warp per 32-source word column with incomplete
// sources (every column when the all-pairs rows are requested: each newly
// reached (source, vertex) pair gets its distance d there). Lane b owns
// source 32*w + b.
// Prev (seen-set pull): level d's new pairs are Nc & ~Prev (S_d & ~S_{d-1});
// NULL: Nc holds them.
__device__ void phase_extract(const MsbfsArgs& a, const uint32_t* Nc, const uint32_t* Prev, int d) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int Wv = (a.nb + 31) >> 5;
    const bool ap = a.apsp != nullptr;
    for (long long w = warp; w < Wv; w += nwarps) {
        const uint32_t need0 = ld_volatile_u32(a.need + w);
        if (need0 == 0u && !ap) continue;
        const long long j = w * 32 + lane;
        const bool mine_need = (need0 >> lane) & 1u;
        int c = mine_need ? __ldcg(a.cnt + j) : a.k;
        bool found = false;
        uint32_t needw = need0;
        int32_t* oi = a.out_idx + (size_t)j * a.k;
        uint16_t* od = a.out_dist + (size_t)j * a.k;
        // eight 32-vertex tiles per round, their loads issued together
        for (int v00 = 0; v00 < a.n && (needw != 0u || ap); v00 += 256) {
            uint32_t xs[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int v = v00 + 32 * q + lane;
                xs[q] = (v < a.n) ? __ldcg(Nc + (size_t)v * a.W + w) : 0u;
                if (Prev && v < a.n) xs[q] &= ~__ldcg(Prev + (size_t)v * a.W + w);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                // a lane whose source needs no entries has c == k and appends none
                const uint32_t x = ap ? xs[q] : (xs[q] & needw);
                // transpose the 32x32 tile with one ballot per source that has
                // a vertex in it (the OR over the lanes lists those sources)
                uint32_t cols = __reduce_or_sync(kFull, x);
                if (cols == 0u) continue;
                uint32_t mine = 0u;
                while (cols) {
                    const int b = __ffs(cols) - 1;
                    cols &= cols - 1u;
                    const uint32_t t = __ballot_sync(kFull, (x >> b) & 1u);
                    if (lane == b) mine = t;
                }
                if (mine) found = true;
                const int v0 = v00 + 32 * q;
                if (ap && mine) {
                    uint16_t* row = a.apsp + (size_t)j * a.apsp_ld + v0;
                    for (uint32_t m = mine; m; m &= m - 1u) row[__ffs(m) - 1] = (uint16_t)d;
                }
                while (mine && c < a.k) {
                    const int i = __ffs(mine) - 1;
                    mine &= mine - 1u;
                    oi[c] = v0 + i;
                    od[c] = (uint16_t)d;
                    ++c;
                }
                needw = __ballot_sync(kFull, mine_need && c < a.k);
            }
        }
        // a source is finished when its list is full or its BFS ran dry
        const bool done = mine_need && (c >= a.k || !found);
        const uint32_t done_mask = __ballot_sync(kFull, done);
        if (mine_need) a.cnt[j] = c;
        if (lane == 0 && done_mask) {
            a.need[w] = need0 & ~done_mask;
            // partial form: a finished source stops propagating
            if (a.partial) a.act[w] = __ldcg(a.act + w) & ~done_mask;
            atomicSub(&a.ctr->n_need, __popc(done_mask));
        }
    }
}

// Thread 0: start the bulk copies of this CTA's staged slice (see
// MsbfsArgs) into dyn, completing on bar. st: [0] positions P, [1] index of
// position p0 among the copied pairs, [2] ocol index of the first copied
// id, [3] 1 if the copies were issued, [4] bytes of the pairs.
__device__ void stage_issue(const MsbfsArgs& a, unsigned long long* bar, int* st, unsigned char* dyn) {
    const int p0 = __ldg(a.slice + blockIdx.x), p1 = __ldg(a.slice + blockIdx.x + 1);
    const int m_lo = p0 & ~1, m_hi = (p1 + 2) & ~1;
    const int c0 = __ldg(&a.meta[p0].y), c1 = __ldg(&a.meta[p1].y);
    const int c_lo = c0 & ~3, c_hi = (c1 + 3) & ~3;
    const long long mb = (long long)(m_hi - m_lo) * 8, cb = (long long)(c_hi - c_lo) * 4;
    st[0] = p1 - p0;
    st[1] = p0 - m_lo;
    st[2] = c_lo;
    st[3] = 0;
    st[4] = (int)mb;
    mbar_init(bar, 1);
    if (a.staged == 2) return;  // test mode: no copies, the slice is read from global memory
    if (p1 >= p0 && cb >= 0 && mb + cb <= a.stage_bytes) {
        mbar_expect_tx(bar, (unsigned)(mb + cb));
        bulk_copy_g2s(dyn, a.meta + m_lo, (unsigned)mb, bar);
        if (cb > 0) bulk_copy_g2s(dyn + mb, a.ocol + c_lo, (unsigned)cb, bar);
        st[3] = 1;
    } else {
        atomicExch(&a.ctr->status, kStatusInternal);  // the host's slice check disagrees with the data
    }
}

// All levels of one launch. copies_done: the staged slice's copies (if any
// were issued) have landed, so the CTA may exit.
template <int GW, int NB, bool STAGED, bool SO>
__device__ __forceinline__ void msbfs_levels(const MsbfsArgs& a, unsigned long long* bar, const int* st,
                                             unsigned char* dyn, bool& copies_done) {
    // phase times of block 0's thread 0, kept in shared memory (not in
    // registers every thread would carry through every phase)
    __shared__ unsigned long long s_time[6];  // last stamp, init, pull, extract, push, push levels
    enum { kLast, kInit, kPull, kExtract, kPush, kPushes };
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    if (timer) {
        s_time[kLast] = globaltimer_ns();
        for (int i = 1; i < 6; ++i) s_time[i] = 0ull;
    }
    auto lap = [&](int slot) {
        if (timer) {
            const unsigned long long t = globaltimer_ns();
            s_time[slot] += t - s_time[kLast];
            s_time[kLast] = t;
        }
    };
    if (a.identity) {
        phase_init_identity<SO>(a);
        if (!grid_barrier(&a.ctr->bar, &a.ctr->status)) return;
    } else {
        phase_init(a);
        if (!grid_barrier(&a.ctr->bar, &a.ctr->status)) return;
        phase_seed(a);
        if (!grid_barrier(&a.ctr->bar, &a.ctr->status)) return;
    }
    StageView sv{nullptr, nullptr, 0, 0, 0};
    if (STAGED) {
        const bool issued = st[3] != 0;
        const bool ok = __syncthreads_and(issued && mbar_wait_bounded(bar, 0, kWaitLimitNs));
        copies_done = ok || !issued;
        if (ok) {
            sv.meta = reinterpret_cast<const int2*>(dyn) + st[1];
            sv.col = reinterpret_cast<const int32_t*>(dyn + st[4]);
            sv.cbase = st[2];
            sv.mode = 1;
        } else {
            if (threadIdx.x == 0 && issued) atomicExch(&a.ctr->status, kStatusTimeout);
            sv.meta = a.meta + __ldg(a.slice + blockIdx.x);
            sv.col = a.ocol;
            sv.cbase = 0;
            sv.mode = 2;
        }
        sv.P = st[0];
    }
    lap(kInit);

    uint32_t* Fc = a.N;  // level-1 frontier was pushed into N
    uint32_t* Nc = a.F;
    // seen-set pull: S_d in buffer d % 3 of {F, N, S}
    auto buf = [&](int i) -> uint32_t* {
        const int r = i % 3;
        return r == 0 ? a.F : (r == 1 ? a.N : a.S);
    };
    int last = 1;
    bool go = ld_volatile_u32(&a.ctr->lvl_any[1]) != 0u;
    if (a.partial && ld_volatile_i32(&a.ctr->n_need) == 0) go = false;
    int last_pull = 0;  // u_edges[0] holds the "everything unvisited" estimate
    // The extraction of level d runs in the same phase as the next level's
    // pull (or push preparation): both only read level d's buffer (now the
    // frontier Fc), so one grid barrier per level is saved. In the partial
    // form the extraction also retires finished sources from act while that
    // pull reads act; a pull that still sees a retired source propagates it
    // one level more, which changes no list (the source's list is final).
    int pend = 0;  // level whose extraction is still to run (0: none)
    for (int d = 2; go && d <= a.n; ++d) {
        const int need_now = ld_volatile_i32(&a.ctr->n_need);
        if (need_now == 0 && !a.apsp) pend = 0;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            // slots of level d + 1 (last used by level d - 3)
            a.ctr->lvl_any[(d + 1) % 3] = 0u;
            a.ctr->qcnt[(d + 1) % 4] = 0;
            a.ctr->f_edges[(d + 1) % 4] = 0ull;
            a.ctr->u_edges[(d + 1) % 4] = 0ull;
            a.ctr->sat_items[(d + 1) % 4] = 0ull;
        }
        // Direction of level d, decided identically by every thread from
        // values settled before the last barrier: push when the edges out of
        // the frontier are few against the edges still to be explored
        // (Beamer's rule in bit-parallel form). The estimate of unexplored
        // edges comes from a pull at most two levels back; older, pull again.
        bool push = false;
        if (SO) {  // the seen-set pull runs pull-only levels
        } else if (a.direction == 2) {
            push = true;
        } else if (a.direction == 0 && d - last_pull <= 2) {
            const unsigned long long fe = *reinterpret_cast<volatile unsigned long long*>(&a.ctr->f_edges[(d - 1) % 4]);
            const unsigned long long ue = *reinterpret_cast<volatile unsigned long long*>(&a.ctr->u_edges[last_pull % 4]);
            push = fe * (unsigned long long)a.push_div < ue;
        }
        bool all_sat = false;
        if (push) {
            phase_push_prep(a, Fc, Nc, d);
            if (pend) phase_extract(a, Fc, nullptr, pend);
            if (!grid_barrier(&a.ctr->bar, &a.ctr->status)) return;
            phase_push(a, Fc, Nc, d);
            if (!grid_barrier(&a.ctr->bar, &a.ctr->status)) return;
            lap(kPush);
            if (timer) ++s_time[kPushes];
        } else {
            if (SO) {
                phase_pull<GW, NB, STAGED, true>(a, buf(d - 1), buf(d), d % 3, d, sv);
                if (pend) phase_extract(a, buf(pend), buf(pend - 1), pend);
            } else {
                phase_pull<GW, NB, STAGED, false>(a, Fc, Nc, d % 3, d, sv);
                if (pend) phase_extract(a, Fc, nullptr, pend);
            }
            if (!grid_barrier(&a.ctr->bar, &a.ctr->status)) return;
            lap(kPull);
            last_pull = d;
            all_sat = !a.partial && *reinterpret_cast<volatile unsigned long long*>(&a.ctr->sat_items[d % 4]) ==
                                        (unsigned long long)a.n * (unsigned long long)(a.W / GW);
        }
        pend = 0;
        if (ld_volatile_u32(&a.ctr->lvl_any[d % 3]) == 0u) break;
        last = d;
        if (a.partial && ld_volatile_i32(&a.ctr->n_need) == 0) break;
        pend = d;
        uint32_t* t = Fc;
        Fc = Nc;
        Nc = t;
        // every active source has reached every vertex: level d + 1 would find
        // nothing, so only the extraction of level d remains (after the loop)
        if (all_sat) break;
    }
    if (pend) {  // every item saturated (or the loop ran out of levels) with an extraction pending
        phase_extract(a, SO ? buf(pend) : Fc, SO ? buf(pend - 1) : nullptr, pend);
        if (!grid_barrier(&a.ctr->bar, &a.ctr->status)) return;
        lap(kExtract);
    }
    if (timer) {
        a.ctr->levels = last;
        a.ctr->level_sum += last;
        if (last > a.ctr->levels_max) a.ctr->levels_max = last;
        a.ctr->t_init_ns += s_time[kInit];
        a.ctr->t_pull_ns += s_time[kPull];
        a.ctr->t_extract_ns += s_time[kExtract];
        a.ctr->t_push_ns += s_time[kPush];
        a.ctr->push_levels += (long long)s_time[kPushes];
    }
}

// OCC: resident CTAs per SM the kernel is built for (3: up to 80 registers a
// thread; 4: 64 registers, more warps to hide latency). STAGED: the light
// rows come from the CTA's slice staged in shared memory (a separate build,
// so the other one carries none of its code or registers).
template <int GW, int OCC, bool STAGED, bool SO>
__global__ void __launch_bounds__(256, OCC) msbfs_kernel(MsbfsArgs a) {
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ int s_stage[5];
    extern __shared__ __align__(16) unsigned char s_dyn[];
    if (STAGED && threadIdx.x == 0) stage_issue(a, &s_bar, s_stage, s_dyn);
    bool copies_done = !STAGED;
    // eight neighbour loads in flight per light item (fewer measured slower even where the
    // 64-register build spills)
    msbfs_levels<GW, 8, STAGED, SO>(a, &s_bar, s_stage, s_dyn, copies_done);
    // a CTA that left early must not exit while a bulk copy still writes its shared memory
    if (STAGED && !copies_done && s_stage[3]) mbar_wait_bounded(&s_bar, 0, kWaitLimitNs);
}

// Self-test of the bounded wait: every CTA but `absent` enters the grid
// barrier, which therefore can never complete; the waiters must give up
// after limit_ns and record kStatusTimeout. No fault, no trap, no hang.
__global__ void barrier_selftest_kernel(GridBarrier* bar, int32_t* status, unsigned long long limit_ns,
                                        int absent) {
    if ((int)blockIdx.x == absent) return;
    grid_barrier(bar, status, limit_ns);
}

// ocol[meta[p].y ...] = the CSR row of vertex meta[p].x, one warp per position.
__global__ void gather_rows_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   const int32_t* __restrict__ heavy, const int2* __restrict__ meta, int32_t n_pos,
                                   int32_t* __restrict__ ocol) {
    const int lane = threadIdx.x & 31;
    for (long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_pos;
         p += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int2 m = meta[p];
        int e0, e1;
        if (m.x >= 0) {
            e0 = row_ptr[m.x];
            e1 = row_ptr[m.x + 1];
        } else {  // segment s of heavy vertex heavy[h]
            const int h = ~m.x / kHubSegMax, sg = ~m.x % kHubSegMax;
            const int v = heavy[h];
            const int r0 = row_ptr[v], r1 = row_ptr[v + 1];
            const int len = hub_seg_len(r1 - r0);
            e0 = r0 + sg * len;
            e1 = min(r1, e0 + len);
        }
        for (int e = e0 + lane; e < e1; e += 32) ocol[m.y + (e - e0)] = col[e];
    }
}

__global__ void identity_kernel(int32_t* dst, int32_t n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (int32_t)i;
}

}  // namespace

namespace {

template <bool STAGED, bool SO>
const void* msbfs_kernel_for_t(int pull_width, int ctas_per_sm) {
    if (pull_width == 2)
        return ctas_per_sm == 4 ? (const void*)msbfs_kernel<2, 4, STAGED, SO>
                                : (const void*)msbfs_kernel<2, 3, STAGED, SO>;
    return ctas_per_sm == 4 ? (const void*)msbfs_kernel<4, 4, STAGED, SO> : (const void*)msbfs_kernel<4, 3, STAGED, SO>;
}

const void* msbfs_kernel_for(int pull_width, int ctas_per_sm, bool staged, bool seen_only) {
    if (seen_only)
        return staged ? msbfs_kernel_for_t<true, true>(pull_width, ctas_per_sm)
                      : msbfs_kernel_for_t<false, true>(pull_width, ctas_per_sm);
    return staged ? msbfs_kernel_for_t<true, false>(pull_width, ctas_per_sm)
                  : msbfs_kernel_for_t<false, false>(pull_width, ctas_per_sm);
}

}  // namespace

// Resident CTAs per SM of a build: the smaller over its two schemes, so one
// cooperative grid size serves both.
int msbfs_max_blocks_per_sm(int block_threads, int pull_width, int ctas_per_sm, size_t dyn_smem, bool staged) {
    int best = 1 << 30;
    for (bool so : {false, true}) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, msbfs_kernel_for(pull_width, ctas_per_sm, staged, so),
                                                          block_threads, dyn_smem) != cudaSuccess)
            return 0;
        best = std::min(best, nb);
    }
    return best;
}

cudaError_t msbfs_allow_smem(int bytes) {
    for (int w : {2, 4})
        for (int c : {3, 4})
            for (bool so : {false, true}) {
                cudaError_t e = cudaFuncSetAttribute(msbfs_kernel_for(w, c, true, so),
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

cudaError_t launch_gather_rows(const int32_t* row_ptr, const int32_t* col, const int32_t* heavy, const int2* meta,
                               int32_t n_pos, int32_t* ocol, cudaStream_t s) {
    if (n_pos <= 0) return cudaSuccess;
    long long g = ((long long)n_pos * 32 + 255) / 256;
    if (g > device_sm_count() * 16ll) g = device_sm_count() * 16ll;
    gather_rows_kernel<<<(unsigned)g, 256, 0, s>>>(row_ptr, col, heavy, meta, n_pos, ocol);
    return cudaGetLastError();
}

// CTAs for one launch: one thread per (vertex, group) item and one warp
// per extraction column, at most the resident maximum. Fewer CTAs make
// every grid barrier cheaper on small graphs.
int msbfs_grid_for(const MsbfsArgs& a, int max_grid) {
    const long long items = (long long)a.n * (a.W >> 2);
    long long g = (items + 255) / 256;
    const long long for_extract = ((a.nb + 31) / 32 + 7) / 8;
    if (g < for_extract) g = for_extract;
    if (g < 1) g = 1;
    if (g > max_grid) g = max_grid;
    return (int)g;
}

cudaError_t launch_msbfs(const MsbfsArgs& a, int grid, int block, cudaStream_t s) {
    MsbfsArgs copy = a;
    void* params[] = {&copy};
    return cudaLaunchCooperativeKernel(msbfs_kernel_for(a.pull_width, a.ctas_per_sm, a.staged != 0, a.seen_only != 0),
                                       dim3(grid), dim3(block), params, a.staged ? (size_t)a.stage_bytes : 0, s);
}

cudaError_t launch_barrier_selftest(GridBarrier* bar, int32_t* status, unsigned long long limit_ns, int grid,
                                    cudaStream_t s) {
    int absent = 0;
    void* params[] = {&bar, &status, &limit_ns, &absent};
    return cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, dim3(grid), dim3(256), params, 0, s);
}

cudaError_t launch_identity(int32_t* dst, int32_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    identity_kernel<<<grid, 256, 0, s>>>(dst, n);
    return cudaGetLastError();
}

}  // namespace gumap
