// Batched engine: many independent graphs (a disjoint union) in one
// persistent launch.
//
// The batch is cut into units (graph g, a block of up to 32*W of its
// sources). Each CTA takes units from an atomic queue and runs the whole
// multi-source BFS of a unit by itself: the frontier and next bitsets of the
// unit's graph live in the CTA's shared memory (and the visited bitset too
// when it fits, otherwise in a CTA-private slab of global memory), so a BFS
// level costs one __syncthreads instead of a grid barrier and the neighbour
// gathers are shared-memory loads. Units of 4 or more words pull 128-bit
// groups (a vertex's neighbour ids are then read once per 4 words). The
// per-level work is the same as the
// global engine (msbfs.cu): a pull N[v] = OR_{u in adj(v)} F[u] masked by
// act & ~visited, with the early exit once every missing source bit is
// covered (frontier expansion of Algorithm 4 / the BFS of Algorithm 1), and
// an extraction that appends each incomplete source's new vertices in id
// order until it holds k (the (distance, id) order of Section 3.3.1).
// Each unit carries the form of its graph: partial units retire a source
// once its list is complete, full units run until no source advances.
//
// Extraction is split over all warps of the CTA: every (word column, vertex
// chunk) pair first counts, per source, its new vertices (32x32 bit tiles
// transposed with ballots), the counts are prefix-summed over the chunks,
// then each pair writes its vertices at the resulting offsets up to k.
#include "gumap_internal.cuh"

namespace gumap {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;

__global__ void __launch_bounds__(kThreads, 1) batch_kernel(BatchArgs a) {
    extern __shared__ uint32_t sm[];
    __shared__ int s_unit;
    __shared__ int s_need;
    __shared__ int s_any;
    __shared__ int cntc[kMaxBatchW][32];  // per extraction item (column, chunk), per lane: new vertices
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    long long level_sum = 0;
    int level_max = 0;
    for (;;) {
        if (tid == 0) s_unit = atomicAdd(a.next_unit, 1);
        __syncthreads();
        const int ui = s_unit;
        if (ui >= a.n_units) break;
        const BatchUnit U = a.units[ui];
        const int n = U.n, W = U.W, nb = U.nb, k = a.k, v0 = U.v0;
        const int nW = n * W;
        uint32_t* Fc = sm;
        uint32_t* Nc = sm + nW;
        uint32_t* V = U.v_global ? a.vslab + (size_t)blockIdx.x * a.vslab_words : sm + 2 * nW;
        uint32_t* act = sm + (U.v_global ? 2 : 3) * nW;
        uint32_t* need = act + W;
        int32_t* cnt = reinterpret_cast<int32_t*>(need + W);
        const long long row0 = (long long)v0 + U.s_lo;  // output row of the unit's source 0

        // ---- init
        for (int i = tid; i < nW; i += kThreads) {
            V[i] = 0u;
            Nc[i] = 0u;
        }
        for (int i = tid; i < W; i += kThreads) {
            const int lo = i * 32;
            const uint32_t m = lo + 32 <= nb ? kFull : (lo >= nb ? 0u : (1u << (nb - lo)) - 1u);
            act[i] = m;
            need[i] = m;
        }
        for (int i = tid; i < nb; i += kThreads) cnt[i] = 0;
        for (long long i = tid; i < (long long)nb * k; i += kThreads) {
            a.out_idx[row0 * k + i] = -1;
            a.out_dist[row0 * k + i] = kDistInf;
        }
        if (tid == 0) {
            s_need = nb;
            s_any = 0;
        }
        __syncthreads();

        // ---- level 0 (sources) and level 1 (push from the sources' rows)
        for (int j = tid; j < nb; j += kThreads) atomicOr(&V[(U.s_lo + j) * W + (j >> 5)], 1u << (j & 31));
        for (int j = warp; j < nb; j += kWarps) {
            const int gs = v0 + U.s_lo + j;
            const int e0 = __ldg(a.row_ptr + gs), e1 = __ldg(a.row_ptr + gs + 1);
            const int deg = e1 - e0;
            const uint32_t bit = 1u << (j & 31);
            for (int e = e0 + lane; e < e1; e += 32) atomicOr(&Nc[(__ldg(a.col + e) - v0) * W + (j >> 5)], bit);
            const int take = deg < k ? deg : k;
            for (int t = lane; t < take; t += 32) {
                a.out_idx[(row0 + j) * k + t] = __ldg(a.col + e0 + t);
                a.out_dist[(row0 + j) * k + t] = 1;
            }
            if (lane == 0) {
                cnt[j] = take;
                if (deg > 0) s_any = 1;
                if (take >= k || deg == 0) {
                    atomicAnd(&need[j >> 5], ~bit);
                    if (U.partial || deg == 0) atomicAnd(&act[j >> 5], ~bit);
                    atomicSub(&s_need, 1);
                }
            }
        }
        __syncthreads();
        int last = 1;
        bool go = s_any != 0 && !(U.partial && s_need == 0);
        {
            uint32_t* t = Fc;  // level 1 sits in Nc
            Fc = Nc;
            Nc = t;
        }
        const int Wv = (nb + 31) >> 5;
        for (int d = 2; go && d <= n; ++d) {
            const int need_now = s_need;
            // ---- pull
            int any = 0;
            if ((W & 3) == 0) {  // 128-bit items: a vertex's neighbour ids read once per 4 words
                const int G4 = W >> 2;
                const uint4* F4 = reinterpret_cast<const uint4*>(Fc);
                uint4* N4 = reinterpret_cast<uint4*>(Nc);
                uint4* V4 = reinterpret_cast<uint4*>(V);
                const uint4* A4 = reinterpret_cast<const uint4*>(act);
                for (int t = tid; t < n * G4; t += kThreads) {
                    const int v = t / G4;
                    const int g = t - v * G4;
                    const uint4 f0 = F4[t], v4 = V4[t], am = A4[g];
                    const uint4 vis = make_uint4(v4.x | f0.x, v4.y | f0.y, v4.z | f0.z, v4.w | f0.w);
                    const uint4 todo = make_uint4(am.x & ~vis.x, am.y & ~vis.y, am.z & ~vis.z, am.w & ~vis.w);
                    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
                    if (todo.x | todo.y | todo.z | todo.w) {
                        const int e0 = __ldg(a.row_ptr + v0 + v), e1 = __ldg(a.row_ptr + v0 + v + 1);
                        for (int e = e0; e < e1; e += 4) {
                            int u[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) u[q] = e + q < e1 ? __ldg(a.col + e + q) - v0 : -1;
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                if (u[q] >= 0) {
                                    const uint4 x = F4[u[q] * G4 + g];
                                    acc.x |= x.x;
                                    acc.y |= x.y;
                                    acc.z |= x.z;
                                    acc.w |= x.w;
                                }
                            if (((acc.x & todo.x) == todo.x) && ((acc.y & todo.y) == todo.y) &&
                                ((acc.z & todo.z) == todo.z) && ((acc.w & todo.w) == todo.w))
                                break;
                        }
                        acc = make_uint4(acc.x & todo.x, acc.y & todo.y, acc.z & todo.z, acc.w & todo.w);
                    }
                    N4[t] = acc;
                    V4[t] = vis;
                    any |= (acc.x | acc.y | acc.z | acc.w) != 0u;
                }
            } else
            for (int t = tid; t < nW; t += kThreads) {
                const int v = t / W;
                const int w = t - v * W;
                const uint32_t vis = V[t] | Fc[t];
                const uint32_t todo = act[w] & ~vis;
                uint32_t acc = 0u;
                if (todo) {
                    const int e0 = __ldg(a.row_ptr + v0 + v), e1 = __ldg(a.row_ptr + v0 + v + 1);
                    for (int e = e0; e < e1; e += 4) {
                        int u[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) u[q] = e + q < e1 ? __ldg(a.col + e + q) - v0 : -1;
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (u[q] >= 0) acc |= Fc[u[q] * W + w];
                        if ((acc & todo) == todo) break;
                    }
                    acc &= todo;
                }
                Nc[t] = acc;
                V[t] = vis;
                any |= acc != 0u;
            }
            if (!__syncthreads_or(any)) break;
            last = d;
            if (need_now > 0) {
                // ---- extraction: warp items (column w, vertex chunk c)
                const int C = Wv < kWarps ? kWarps / Wv : 1;  // chunks per column
                const int items = Wv * C;
                const int tiles = (n + 31) >> 5;
                const int per = (tiles + C - 1) / C;
                for (int pass = 0; pass < 2; ++pass) {
                    for (int it = warp; it < items; it += kWarps) {
                        const int w = it / C, c = it - w * C;
                        const uint32_t needw = need[w];
                        const int j = w * 32 + lane;
                        const bool mine = (needw >> lane) & 1u;
                        int pos = k;  // sources not in need write nothing
                        if (pass == 1 && mine) {
                            pos = cnt[j];
                            for (int c2 = 0; c2 < c; ++c2) pos += cntc[w * C + c2][lane];
                        }
                        int counted = 0;
                        for (int tl = c * per; tl < (c + 1) * per && tl < tiles; ++tl) {
                            const int v = tl * 32 + lane;
                            const uint32_t x = (v < n ? Nc[v * W + w] : 0u) & needw;
                            // one ballot per source with a vertex in the tile
                            uint32_t cols = __reduce_or_sync(kFull, x);
                            if (cols == 0u) continue;
                            uint32_t m = 0u;
                            while (cols) {
                                const int b = __ffs(cols) - 1;
                                cols &= cols - 1u;
                                const uint32_t tb = __ballot_sync(kFull, (x >> b) & 1u);
                                if (lane == b) m = tb;
                            }
                            if (pass == 0) {
                                counted += __popc(m);
                            } else {
                                while (m && pos < k) {
                                    const int i = __ffs(m) - 1;
                                    m &= m - 1u;
                                    a.out_idx[(row0 + j) * k + pos] = v0 + tl * 32 + i;
                                    a.out_dist[(row0 + j) * k + pos] = (uint16_t)d;
                                    ++pos;
                                }
                            }
                        }
                        if (pass == 0) cntc[it][lane] = counted;
                    }
                    __syncthreads();
                }
                // ---- bookkeeping: new counts, finished sources
                for (int w = warp; w < Wv; w += kWarps) {
                    const uint32_t needw = need[w];
                    const int j = w * 32 + lane;
                    const bool mine = (needw >> lane) & 1u;
                    int found = 0;
                    for (int c = 0; c < C; ++c) found += cntc[w * C + c][lane];
                    int c_new = mine ? cnt[j] + found : 0;
                    if (c_new > k) c_new = k;
                    const bool done = mine && (c_new >= k || found == 0);
                    const uint32_t done_mask = __ballot_sync(kFull, done);
                    if (mine) cnt[j] = c_new;
                    if (lane == 0 && done_mask) {
                        need[w] = needw & ~done_mask;
                        if (U.partial) act[w] &= ~done_mask;
                        atomicSub(&s_need, __popc(done_mask));
                    }
                }
                __syncthreads();
                if (U.partial && s_need == 0) break;
            }
            uint32_t* t = Fc;
            Fc = Nc;
            Nc = t;
        }
        level_sum += last;
        if (last > level_max) level_max = last;
        // the unit's bytes on the model of the global engine: per level the
        // frontier, visited and next rows of n vertices and W words (here in
        // shared memory) plus the graph's CSR
        if (tid == 0) {
            const unsigned long long nnz_g =
                (unsigned long long)(__ldg(a.row_ptr + v0 + n) - __ldg(a.row_ptr + v0));
            atomicAdd(&a.ctr->model_bytes, (unsigned long long)last * (12ull * (unsigned long long)n * W +
                                                                      4ull * (unsigned long long)(n + 1) + 4ull * nnz_g));
        }
        __syncthreads();  // the next unit reuses shared memory
    }
    if (tid == 0 && level_sum) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.ctr->level_sum), (unsigned long long)level_sum);
        atomicMax(&a.ctr->levels_max, level_max);
    }
}

}  // namespace

cudaError_t batch_prepare(size_t smem_bytes) {
    return cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

int batch_threads() { return kThreads; }

const void* batch_kernel_ptr() { return (const void*)batch_kernel; }

cudaError_t launch_batch(const BatchArgs& a, int grid, size_t smem_bytes, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.next_unit, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    batch_kernel<<<grid, kThreads, smem_bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gumap
