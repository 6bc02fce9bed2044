// Partial form (PartialBFS, Algorithm 4): one BFS per source, stopped after
// the level at which k other vertices have been reached.
//
// The source's BFS proceeds level by level. The candidates of level d are
// the neighbours of the level d-1 vertices; because every CSR row is sorted,
// they can be enumerated in ascending id by merging those rows: each round
// takes the minimum head, advances every row whose head equals it, and keeps
// the id if it is new. A neighbour of a level d-1 vertex lies at level d-2,
// d-1 or d, so "new" is a check against the levels d-2 and d-1 only; both
// were emitted in ascending id, and the candidates of level d come out in
// ascending id, so two pointers that only move forward decide membership.
// The merge stops as soon as the list holds k entries; since ids come out in
// ascending order, those are the k smallest by (distance, id), and no
// adjacency beyond that point is read. A level that yields nothing ends the
// search (the component is exhausted) and the rest of the row is padding.
//
// Every level before the last yields fewer than k new vertices, so the
// frontier never holds more than k - 1 rows.
//
// Three builds of that merge (GUMAP_OPT_FRONTIER_BUILD; the autotuner times
// them on the handle's graph):
//   GROUP (default): a group of G lanes per source, G = 4 for k <= 17, 8 for
//     k <= 65, 16 for k <= 129, else 32; a lane owns frontier rows, the
//     minimum is a shuffle reduction within the group, and all groups of a
//     warp run one flat loop (see frontier_group_kernel). A warp-wide merge
//     spends its whole issue slot on one candidate of one source; a group of
//     G lanes shares it among 32 / G sources.
//   THREAD (k <= 64): one thread per source; its list, the frontier rows'
//     cursors and heads live in shared memory (element q of thread t at
//     q * T + t, so a warp reading the same element hits 32 banks). Fewest
//     instructions per candidate, but the state limits the threads per SM.
//   WARP: one warp per source, one frontier row per lane (several per lane
//     beyond 32 rows), the minimum taken by a warp reduction.
#include "gumap_internal.cuh"

#include <climits>

namespace gumap {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;

template <int LPL>
__global__ void __launch_bounds__(kThreads) frontier_kernel(FrontierArgs a) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int32_t* lst = smem + wib * (a.k + 1);  // lst[0] = source, lst[1 + t] = t-th found vertex
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long j = warp; j < a.n_src; j += nwarps) {
        const int s = a.src ? a.src[j] : (int)j;
        int32_t* oi = a.out_idx + (size_t)j * a.k;
        uint16_t* od = a.out_dist + (size_t)j * a.k;
        if (s < 0 || s >= a.n) {  // an invalid source is an empty row
            if (lane == 0) atomicExch(a.status, kStatusBadSource);
            for (int t = lane; t < a.k; t += 32) {
                oi[t] = -1;
                od[t] = kDistInf;
            }
            continue;
        }
        if (lane == 0) lst[0] = s;
        __syncwarp();
        int c = 0;              // vertices found so far
        int fs = 0, fe = 1;     // frontier = lst[fs, fe) (level d-1)
        int chk = 1;            // visited check range lst[chk, lvl_start) = levels d-2, d-1
        for (int d = 1;; ++d) {
            const int nf = fe - fs;
            int p[LPL], e[LPL], h[LPL];
#pragma unroll
            for (int q = 0; q < LPL; ++q) {
                const int r = lane + 32 * q;
                h[q] = INT_MAX;
                p[q] = 0;
                e[q] = 0;
                if (r < nf) {
                    const int u = lst[fs + r];
                    p[q] = __ldg(a.row_ptr + u);
                    e[q] = __ldg(a.row_ptr + u + 1);
                    if (p[q] < e[q]) h[q] = __ldg(a.col + p[q]);
                }
            }
            const int lvl_start = 1 + c;
            int found = 0;
            while (c < a.k) {
                int lm = INT_MAX;
#pragma unroll
                for (int q = 0; q < LPL; ++q) lm = min(lm, h[q]);
                const int m = __reduce_min_sync(kFull, lm);
                if (m == INT_MAX) break;
#pragma unroll
                for (int q = 0; q < LPL; ++q) {
                    if (h[q] == m) {
                        ++p[q];
                        h[q] = p[q] < e[q] ? __ldg(a.col + p[q]) : INT_MAX;
                    }
                }
                bool hit = false;
                for (int t = chk + lane; t < lvl_start; t += 32) hit |= (lst[t] == m);
                if (__any_sync(kFull, hit)) continue;
                if (lane == 0) {
                    lst[1 + c] = m;
                    oi[c] = m;
                    od[c] = (uint16_t)d;
                }
                ++c;
                ++found;
                __syncwarp();
            }
            if (c >= a.k || found == 0) break;
            chk = fs;  // level d-1 becomes level d-2 of the next round
            fs = lvl_start;
            fe = 1 + c;
        }
        for (int t = c + lane; t < a.k; t += 32) {
            oi[t] = -1;
            od[t] = kDistInf;
        }
        __syncwarp();
    }
}

constexpr int kThreadMaxK = 64;  // largest k of the thread-per-source build

// One thread per source (k <= kThreadMaxK). Shared memory per thread, each
// array strided by the block size T: lst[k + 1] (lst[0] the source, then the
// vertices found, level by level, ascending within a level), and for each
// frontier row (at most k - 1) its cursor, end and current head.
__global__ void __launch_bounds__(128) frontier_thread_kernel(FrontierArgs a) {
    extern __shared__ int32_t fsm[];
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int k = a.k;
    int32_t* lst = fsm + t;                  // lst[i * T]
    int32_t* rpos = fsm + (k + 1) * T + t;   // rpos[q * T]
    int32_t* rend = rpos + k * T;
    int32_t* head = rend + k * T;
    const long long stride = (long long)gridDim.x * T;
    for (long long j = (long long)blockIdx.x * T + t; j < a.n_src; j += stride) {
        const int s = a.src ? a.src[j] : (int)j;
        int32_t* oi = a.out_idx + (size_t)j * k;
        uint16_t* od = a.out_dist + (size_t)j * k;
        int c = 0;  // vertices found so far
        if (s < 0 || s >= a.n) {  // an invalid source is an empty row
            atomicExch(a.status, kStatusBadSource);
        } else {
            lst[0] = s;
            int fs = 0, fe = 1;  // frontier = lst[fs, fe) (level d-1)
            int chk = 1;         // level d-2 = lst[chk, fs) (empty at d = 1)
            for (int d = 1;; ++d) {
                const int nf = fe - fs;
                for (int q = 0; q < nf; ++q) {
                    const int u = lst[(fs + q) * T];
                    const int p0 = __ldg(a.row_ptr + u), p1 = __ldg(a.row_ptr + u + 1);
                    rpos[q * T] = p0;
                    rend[q * T] = p1;
                    head[q * T] = p0 < p1 ? __ldg(a.col + p0) : INT_MAX;
                }
                const int lvl_start = 1 + c;
                int pa = chk, pb = fs;  // forward pointers into levels d-2 and d-1
                int found = 0;
                while (c < k) {
                    int m = INT_MAX;
                    for (int q = 0; q < nf; ++q) m = min(m, head[q * T]);
                    if (m == INT_MAX) break;
                    for (int q = 0; q < nf; ++q) {
                        if (head[q * T] == m) {
                            const int p = rpos[q * T] + 1;
                            rpos[q * T] = p;
                            head[q * T] = p < rend[q * T] ? __ldg(a.col + p) : INT_MAX;
                        }
                    }
                    while (pa < fs && lst[pa * T] < m) ++pa;
                    while (pb < fe && lst[pb * T] < m) ++pb;
                    if ((pa < fs && lst[pa * T] == m) || (pb < fe && lst[pb * T] == m)) continue;
                    lst[(1 + c) * T] = m;
                    oi[c] = m;
                    od[c] = (uint16_t)d;
                    ++c;
                    ++found;
                }
                if (c >= k || found == 0) break;
                chk = fs;  // level d-1 becomes level d-2 of the next round
                fs = lvl_start;
                fe = 1 + c;
            }
        }
        for (int q = c; q < k; ++q) {
            oi[q] = -1;
            od[q] = kDistInf;
        }
    }
}

size_t thread_smem_bytes(int k, int threads) { return (size_t)(4 * k + 1) * threads * sizeof(int32_t); }

cudaError_t launch_thread(const FrontierArgs& a, cudaStream_t s) {
    // as many threads per CTA (a multiple of 32, at most 128) as keep the
    // CTA's state within 48 KB
    int threads = 128;
    while (threads > 32 && thread_smem_bytes(a.k, threads) > 48 * 1024) threads -= 32;
    const size_t smem = thread_smem_bytes(a.k, threads);
    long long g = ((long long)a.n_src + threads - 1) / threads;
    const long long cap = (long long)(a.sms > 0 ? a.sms : device_sm_count()) * 64;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    frontier_thread_kernel<<<(unsigned)g, threads, smem, s>>>(a);
    return cudaGetLastError();
}

// One group of G lanes per source (G = 4, 8, 16 or 32, by k), 32 / G sources
// per warp. Lane r of a group owns frontier rows r, r + G, ... (LPL slots).
// Every lane runs the same flat loop; an iteration is one merge round of
// every group in its merge, preceded, when any group needs it, by the
// transitions of the groups that start a source or a level. So the warp's
// collectives always see all 32 lanes, and a group that finishes a level or
// a source does not hold the others back. A group's list is in shared
// memory (lst[0] the source, then the vertices found).
template <int G, int LPL>
__global__ void __launch_bounds__(kThreads) frontier_group_kernel(FrontierArgs a) {
    extern __shared__ int32_t gsm[];
    constexpr int NG = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gi = lane / G;
    const int gl = lane % G;
    const int k = a.k;
    int32_t* lst = gsm + ((threadIdx.x >> 5) * NG + gi) * (k + 1);
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long gstride = nwarps * NG;
    long long j = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * NG + gi;
    int st = 0;  // 0: take source j, 1: load the level's frontier rows, 2: merge, 3: no sources left
    int c = 0, d = 0, fs = 0, fe = 0, chk = 0, lvl = 0, found = 0, pa = 0, pb = 0, qmax = 0;
    int32_t* oi = a.out_idx;
    uint16_t* od = a.out_dist;
    int p[LPL], e[LPL], h[LPL];
#pragma unroll
    for (int q = 0; q < LPL; ++q) {
        p[q] = 0;
        e[q] = 0;
        h[q] = INT_MAX;
    }
    while (true) {
        if (__any_sync(kFull, st < 2)) {
            if (st == 0) {
                if (j >= a.n_src) {
                    st = 3;
                } else {
                    const int s = a.src ? a.src[j] : (int)j;
                    oi = a.out_idx + (size_t)j * k;
                    od = a.out_dist + (size_t)j * k;
                    c = 0;
                    if (s < 0 || s >= a.n) {  // an invalid source is an empty row
                        if (gl == 0) atomicExch(a.status, kStatusBadSource);
                        for (int t = gl; t < k; t += G) {
                            oi[t] = -1;
                            od[t] = kDistInf;
                        }
                        j += gstride;  // the next source, next iteration
                    } else {
                        if (gl == 0) lst[0] = s;
                        d = 0;
                        fs = 0;
                        fe = 1;
                        chk = 1;
                        st = 1;
                    }
                }
            }
            __syncwarp();
            if (st == 1) {
                ++d;
                const int nf = fe - fs;
#pragma unroll
                for (int q = 0; q < LPL; ++q) {
                    const int r = gl + G * q;
                    h[q] = INT_MAX;
                    if (r < nf) {
                        const int u = lst[fs + r];
                        p[q] = __ldg(a.row_ptr + u);
                        e[q] = __ldg(a.row_ptr + u + 1);
                        if (p[q] < e[q]) h[q] = __ldg(a.col + p[q]);
                    }
                }
                lvl = 1 + c;
                pa = chk;
                pb = fs;
                found = 0;
                st = 2;
            }
            // row slots any group of the warp uses at its current level
            const int nfw = __reduce_max_sync(kFull, st == 2 ? fe - fs : 0);
            qmax = (nfw + G - 1) / G;
        }
        if (__all_sync(kFull, st == 3)) break;
        int lm = INT_MAX;
#pragma unroll
        for (int q = 0; q < LPL; ++q)
            if (q < qmax) lm = min(lm, h[q]);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) lm = min(lm, __shfl_xor_sync(kFull, lm, o));
        if (st == 2) {
            if (lm == INT_MAX || c >= k) {  // the level is over
                if (c >= k || found == 0) {  // the list is full, or the component ran out
                    for (int t = c + gl; t < k; t += G) {
                        oi[t] = -1;
                        od[t] = kDistInf;
                    }
                    j += gstride;
                    st = 0;
                } else {
                    chk = fs;  // level d-1 becomes level d-2 of the next round
                    fs = lvl;
                    fe = 1 + c;
                    st = 1;
                }
            } else {
#pragma unroll
                for (int q = 0; q < LPL; ++q) {
                    if (q < qmax && h[q] == lm) {
                        ++p[q];
                        h[q] = p[q] < e[q] ? __ldg(a.col + p[q]) : INT_MAX;
                    }
                }
                while (pa < fs && lst[pa] < lm) ++pa;
                while (pb < fe && lst[pb] < lm) ++pb;
                if (!((pa < fs && lst[pa] == lm) || (pb < fe && lst[pb] == lm))) {
                    if (gl == 0) {
                        lst[1 + c] = lm;
                        oi[c] = lm;
                        od[c] = (uint16_t)d;
                    }
                    ++c;
                    ++found;
                }
            }
        }
        __syncwarp();
    }
}

template <int G, int LPL>
cudaError_t launch_group_t(const FrontierArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)kWarpsPerBlock * (32 / G) * (a.k + 1) * sizeof(int32_t);
    long long g = ((long long)a.n_src + kWarpsPerBlock * (32 / G) - 1) / (kWarpsPerBlock * (32 / G));
    const long long cap = (long long)(a.sms > 0 ? a.sms : device_sm_count()) * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    frontier_group_kernel<G, LPL><<<(unsigned)g, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// Lanes per source by k: the frontier holds at most k - 1 rows (1 at level 1).
cudaError_t launch_group(const FrontierArgs& a, cudaStream_t s) {
    const int maxf = a.k - 1 > 0 ? a.k - 1 : 1;
    if (maxf <= 4) return launch_group_t<4, 1>(a, s);
    if (maxf <= 8) return launch_group_t<4, 2>(a, s);
    if (maxf <= 16) return launch_group_t<4, 4>(a, s);
    if (maxf <= 32) return launch_group_t<8, 4>(a, s);
    if (maxf <= 64) return launch_group_t<8, 8>(a, s);
    if (maxf <= 128) return launch_group_t<16, 8>(a, s);
    return launch_group_t<32, 8>(a, s);
}

template <int LPL>
cudaError_t launch_lpl(const FrontierArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)kWarpsPerBlock * (a.k + 1) * sizeof(int32_t);
    long long g = ((long long)a.n_src + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const long long cap = (long long)(a.sms > 0 ? a.sms : device_sm_count()) * 64;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    frontier_kernel<LPL><<<(unsigned)g, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_frontier(const FrontierArgs& a, cudaStream_t s) {
    if (a.n_src <= 0) return cudaSuccess;
    if (a.build == 0 || a.build == 3) return launch_group(a, s);
    if (a.build == 1 && a.k <= kThreadMaxK) return launch_thread(a, s);
    const int maxf = a.k - 1 > 0 ? a.k - 1 : 1;  // frontier rows at most k - 1 (level 1: the source)
    if (maxf <= 32) return launch_lpl<1>(a, s);
    if (maxf <= 64) return launch_lpl<2>(a, s);
    if (maxf <= 128) return launch_lpl<4>(a, s);
    return launch_lpl<8>(a, s);
}

}  // namespace gumap
