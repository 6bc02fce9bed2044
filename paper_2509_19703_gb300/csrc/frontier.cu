// Partial form (PartialBFS, Algorithm 4) with one warp per source.
//
// The source's BFS proceeds level by level. The candidates of level d are
// the neighbours of the level d-1 vertices; because every CSR row is sorted,
// they can be enumerated in ascending id by merging those rows (one row per
// lane, several per lane for k > 33): each round the warp takes the minimum
// head, advances every row whose head equals it, and keeps the id if it is
// new. A neighbour of a level d-1 vertex lies at level d-2, d-1 or d, so
// "new" is a check against the levels d-2 and d-1 only (kept in shared
// memory). The merge stops as soon as the list holds k entries; since ids
// come out in ascending order, those are the k smallest by (distance, id),
// and no adjacency beyond that point is read. A level that yields nothing
// ends the search (the component is exhausted) and the rest of the row is
// padding.
//
// Every level before the last yields fewer than k new vertices, so the
// frontier never holds more than k - 1 rows: k <= 256 means at most 8 rows
// per lane.
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

template <int LPL>
cudaError_t launch_lpl(const FrontierArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)kWarpsPerBlock * (a.k + 1) * sizeof(int32_t);
    long long g = ((long long)a.n_src + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (g > device_sm_count() * 64ll) g = device_sm_count() * 64ll;
    if (g < 1) g = 1;
    frontier_kernel<LPL><<<(unsigned)g, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_frontier(const FrontierArgs& a, cudaStream_t s) {
    if (a.n_src <= 0) return cudaSuccess;
    const int maxf = a.k - 1 > 0 ? a.k - 1 : 1;  // frontier rows at most k - 1 (level 1: the source)
    if (maxf <= 32) return launch_lpl<1>(a, s);
    if (maxf <= 64) return launch_lpl<2>(a, s);
    if (maxf <= 128) return launch_lpl<4>(a, s);
    return launch_lpl<8>(a, s);
}

}  // namespace gumap
