// UMAP fuzzy weights of the kNN lists (Section 2.1, h_ij) and their fuzzy
// union (the symmetrisation of the UMAP implementation the paper builds on,
// Section 4.1.1).
//
// smooth_knn: one lane per row, 32 rows per warp. The warp stages its rows'
// distances in shared memory (row stride an odd number of words, so the 32
// lanes reading one slot each of their own rows hit 32 different banks);
// then each lane finds rho_i = the smallest valid distance of its row and
// sigma_i solving
//     f(sigma) = sum_j exp(-max(0, d_ij - rho_i)/sigma) = T,  T = log2 k,
// by FP32 bisection on a bracket [0, hi] whose hi doubles until f(hi) >= T.
// Hop distances are integers, so with y = exp(-1/sigma) the sum is the
// polynomial f = sum_L c_L y^(L - rho) over the row's levels L (c_L slots at
// level L); it is evaluated by Horner's rule, on level counts kept in
// registers when the row's levels span fewer than 16, else over the sorted
// row's slots: one exp per bisection step instead of one per slot. f rises strictly from
// c_eq = #{j : d_ij = rho_i} (sigma -> 0) to kv = #valid (sigma -> inf), so
// a root exists iff c_eq < T < kv:
//   kv <= T   -> no root, sigma = +inf, every weight 1;
//   c_eq >= T -> no root, sigma -> 0+, lifted by the floor;
// and sigma = max(sigma*, 1e-3 * mean_j d_ij). Both decisions compare exact
// integers with T, and log2 k is at least 0.0056 away from any integer for a
// k that is not a power of two, so FP32 and FP64 take the same branch.
// Besides rho and sigma each row gets a 16-byte record (WeightRow): rho,
// sigma and the (distance, id) key of its list's last slot.
//
// union: w_ij = a_ij + a_ji - a_ij a_ji with a_ji = 0 when i is not in j's
// list. Hop distances are symmetric, so i can sit in j's list only at
// distance d_ij; and j's list holds the k smallest (distance, id) keys of
// its reachable vertices, so i is in it exactly when the list is not full
// (it then holds every vertex j reaches, i among them) or (d_ij, i) is at
// most the key of its last slot. Both weights are recomputed from the two
// rows' records with the same expression the directed weights use, so the
// union needs one 16-byte record per neighbour and no search of its row.
#include "gumap_internal.cuh"

#include <climits>
#include <math_constants.h>

namespace gumap {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kSkThreads = 128;  // 4 warps, 32 rows each
constexpr int kSkWarps = kSkThreads / 32;

// a_ij = exp(-max(0, d - rho) / sigma) of one valid slot (d >= rho): the one
// expression every kernel evaluates, so that weights of the same slot agree
// bit for bit wherever they are computed.
__device__ __forceinline__ float umap_a(int d, int rho, float sigma) {
    return isinf(sigma) ? 1.0f : expf(-(float)(d - rho) / sigma);
}

// 32-bit words per staged row: enough for k uint16 values, odd.
__host__ __device__ __forceinline__ int sk_stride(int k) { return ((k + 1) / 2) | 1; }

// f(sigma) of one row by Horner's rule over its valid slots d[0 .. kv - 1]
// (ascending distances, d[0] = rho): going down the row, the accumulated
// sum is multiplied by y^(gap) whenever the level drops, then the slot adds
// 1. BFS levels are contiguous, so every gap is 1 (y itself); a wider gap
// costs one more exp.
__device__ __forceinline__ float f_poly(const uint16_t* __restrict__ d, int kv, int rho, float sigma) {
    const float y = expf(-1.0f / sigma);
    float acc = 0.0f;
    int prev = d[kv - 1];
    for (int t = kv - 1; t >= 0; --t) {
        const int x = d[t];
        if (x != prev) {
            const int gap = prev - x;
            acc *= gap == 1 ? y : expf(-(float)gap / sigma);
            prev = x;
        }
        acc += 1.0f;
    }
    if (prev != rho) acc *= expf(-(float)(prev - rho) / sigma);
    return acc;
}

// Rows whose levels span fewer than kLevels keep the count of each level in
// registers: f(sigma) is then the polynomial sum_l c_l y^l, l = 0 .. kLevels - 1,
// by Horner's rule in kLevels multiply-adds.
constexpr int kLevels = 16;

__device__ __forceinline__ float f_levels(const float (&cl)[kLevels], float sigma) {
    const float y = expf(-1.0f / sigma);
    float acc = cl[kLevels - 1];
#pragma unroll
    for (int q = kLevels - 2; q >= 0; --q) acc = acc * y + cl[q];
    return acc;
}

// a: NULL, or [n_rows][k] directed weights (padding 0). rec: NULL, or the
// per-row records for the union (idx then gives the last slot's id).
__global__ void __launch_bounds__(kSkThreads) smooth_knn_kernel(const int32_t* __restrict__ idx,
                                                                const uint16_t* __restrict__ dist, int n_rows,
                                                                int k, float T, float* __restrict__ rho_out,
                                                                float* __restrict__ sigma_out,
                                                                WeightRow* __restrict__ rec, float* __restrict__ a_out) {
    extern __shared__ uint32_t sk_smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int stride = sk_stride(k);
    uint32_t* buf = sk_smem + (size_t)wib * 32 * stride;
    const long long chunks = ((long long)n_rows + 31) / 32;
    for (long long ch = (long long)blockIdx.x * kSkWarps + wib; ch < chunks; ch += (long long)gridDim.x * kSkWarps) {
        const long long r0 = ch * 32;
        const int nr = (int)min(32ll, (long long)n_rows - r0);
        // stage the chunk's rows: slot e of the chunk is row e / k, slot e % k
        const uint16_t* src = dist + r0 * k;
        const int total = nr * k;
        for (int e = lane; e < total; e += 32) {
            const int r = e / k;
            reinterpret_cast<uint16_t*>(buf + r * stride)[e - r * k] = src[e];
        }
        __syncwarp();
        const uint16_t* my = reinterpret_cast<const uint16_t*>(buf + lane * stride);
        int kv = 0, rho = 0;
        float sigma = 0.0f;
        if (lane < nr) {
            while (kv < k && my[kv] != kDistInf) ++kv;
            if (kv > 0) {
                rho = my[0];
                int sum = 0;  // at most 256 values below 2^16
                for (int t = 0; t < kv; ++t) {
                    rho = min(rho, (int)my[t]);
                    sum += my[t];
                }
                int ceq = 0;
                for (int t = 0; t < kv; ++t) ceq += my[t] == rho ? 1 : 0;
                const float mean = (float)sum / (float)kv;
                if ((float)kv <= T) {
                    sigma = CUDART_INF_F;
                } else if ((float)ceq >= T) {
                    sigma = 0.0f;
                } else if ((int)my[kv - 1] - rho < kLevels) {
                    // level counts: the row is sorted, so each level is one run
                    float cl[kLevels];
#pragma unroll
                    for (int q = 0; q < kLevels; ++q) cl[q] = 0.0f;
                    int cur = 0, cnt = 0;
                    for (int t = 0; t < kv; ++t) {
                        const int l = (int)my[t] - rho;
                        if (l != cur) {
#pragma unroll
                            for (int q = 0; q < kLevels; ++q)
                                if (q == cur) cl[q] = (float)cnt;
                            cur = l;
                            cnt = 0;
                        }
                        ++cnt;
                    }
#pragma unroll
                    for (int q = 0; q < kLevels; ++q)
                        if (q == cur) cl[q] = (float)cnt;
                    float lo = 0.0f, hi = 1.0f;
                    for (int it = 0; it < 128 && f_levels(cl, hi) < T; ++it) hi *= 2.0f;
                    for (int it = 0; it < 200; ++it) {
                        const float mid = 0.5f * (lo + hi);
                        if (!(mid > lo && mid < hi)) break;
                        if (f_levels(cl, mid) > T) hi = mid;
                        else lo = mid;
                    }
                    sigma = 0.5f * (lo + hi);
                } else {
                    float lo = 0.0f, hi = 1.0f;
                    for (int it = 0; it < 128 && f_poly(my, kv, rho, hi) < T; ++it) hi *= 2.0f;
                    for (int it = 0; it < 200; ++it) {
                        const float mid = 0.5f * (lo + hi);
                        if (!(mid > lo && mid < hi)) break;
                        if (f_poly(my, kv, rho, mid) > T) hi = mid;
                        else lo = mid;
                    }
                    sigma = 0.5f * (lo + hi);
                }
                sigma = fmaxf(sigma, 1e-3f * mean);
            }
            const long long i = r0 + lane;
            rho_out[i] = (float)rho;
            sigma_out[i] = sigma;
            if (rec) {
                WeightRow wr;
                wr.last_dist = my[k - 1];
                wr.last_id = wr.last_dist == kDistInf ? -1 : __ldg(idx + i * k + (k - 1));
                wr.rho = rho;
                wr.sigma = sigma;
                rec[i] = wr;
            }
        }
        if (a_out) {  // directed weights, one row at a time, coalesced
            for (int r = 0; r < nr; ++r) {
                const int kv_r = __shfl_sync(kFull, kv, r);
                const int rho_r = __shfl_sync(kFull, rho, r);
                const float sg_r = __shfl_sync(kFull, sigma, r);
                const uint16_t* dr = reinterpret_cast<const uint16_t*>(buf + r * stride);
                float* ar = a_out + (r0 + r) * k;
                for (int t = lane; t < k; t += 32) ar[t] = t < kv_r ? umap_a(dr[t], rho_r, sg_r) : 0.0f;
            }
        }
        __syncwarp();
    }
}

// Is row i at distance d in row j's list, whose record is rj?
__device__ __forceinline__ bool in_list(const WeightRow& rj, int i, int d) {
    return rj.last_dist == (int)kDistInf || d < rj.last_dist || (d == rj.last_dist && i <= rj.last_id);
}

// One thread per slot (i, t): union weight into w.
__global__ void __launch_bounds__(256) union_kernel(const int32_t* __restrict__ idx,
                                                    const uint16_t* __restrict__ dist,
                                                    const WeightRow* __restrict__ rec, int n, int k,
                                                    float* __restrict__ w) {
    const long long total = (long long)n * k;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < total;
         s += (long long)gridDim.x * blockDim.x) {
        const long long i = s / k;
        const int j = idx[s];
        float wv = 0.0f;
        if (j >= 0) {
            const int d = dist[s];
            const WeightRow ri = rec[i];
            const WeightRow rj = rec[j];
            const float aij = umap_a(d, ri.rho, ri.sigma);
            const float aji = in_list(rj, (int)i, d) ? umap_a(d, rj.rho, rj.sigma) : 0.0f;
            wv = aij + aji - aij * aji;
        }
        w[s] = wv;
    }
}

// The union weights, plus what the row-by-row COO build (coo.cu) needs: per
// row its valid-slot count (kval), and the mirrors -- slots (i, t) whose
// target j does not list i, so that (j, i) is an entry of row j that j's own
// list lacks -- compacted in slot order as keys (i << 32) | j with the slot's
// weight. One CTA per tile of kUnionTile slots (tile ids from a counter, so
// a tile only waits for tiles handed out before it): chunk c of the tile is
// slots c * 256 + thread, a mirror's place is the mirrors before it in the
// tile (ballots per warp and chunk) plus those of the tiles before (decoupled
// look-back on published per-tile counts). The last tile stores the total.
constexpr int kUnionChunks = 8;
constexpr int kUnionTile = 256 * kUnionChunks;
constexpr unsigned long long kUFlagAggregate = 1ull << 62;
constexpr unsigned long long kUFlagInclusive = 2ull << 62;
constexpr unsigned long long kUCountMask = (1ull << 62) - 1ull;

__device__ __forceinline__ unsigned long long u_globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(256) union_mirrors_kernel(const int32_t* __restrict__ idx,
                                                            const uint16_t* __restrict__ dist,
                                                            const WeightRow* __restrict__ rec, int n, int k,
                                                            float* __restrict__ w, int32_t* __restrict__ kval,
                                                            unsigned long long* __restrict__ mkey,
                                                            float* __restrict__ mval, UnionScan scan) {
    __shared__ unsigned s_tile;
    __shared__ unsigned s_cnt[kUnionChunks][8];
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(scan.tile_ctr, 1u);
    __syncthreads();
    const long long tile = s_tile;
    const long long total = (long long)n * k;
    int jv[kUnionChunks];
    float wv[kUnionChunks];
    unsigned ball[kUnionChunks];
#pragma unroll
    for (int c = 0; c < kUnionChunks; ++c) {
        const long long s = tile * kUnionTile + c * 256 + tid;
        bool mirror = false;
        jv[c] = -1;
        wv[c] = 0.0f;
        if (s < total) {
            const long long i = s / k;
            const int t = (int)(s - i * k);
            const int j = idx[s];
            jv[c] = j;
            if (j >= 0) {
                const int d = dist[s];
                const WeightRow ri = rec[i];
                const WeightRow rj = rec[j];
                const float aij = umap_a(d, ri.rho, ri.sigma);
                const bool mutual = in_list(rj, (int)i, d);
                const float aji = mutual ? umap_a(d, rj.rho, rj.sigma) : 0.0f;
                wv[c] = aij + aji - aij * aji;
                mirror = !mutual;
                if (t == k - 1 || idx[s + 1] < 0) kval[i] = t + 1;
            } else if (t == 0) {
                kval[i] = 0;
            }
            w[s] = wv[c];
        }
        ball[c] = __ballot_sync(0xFFFFFFFFu, mirror);
        if (lane == 0) s_cnt[c][warp] = __popc(ball[c]);
    }
    __syncthreads();
    if (tid == 0) {
        // mirrors of the tile in slot order: chunk by chunk, warp by warp
        unsigned run = 0;
        for (int c = 0; c < kUnionChunks; ++c)
            for (int q = 0; q < 8; ++q) {
                const unsigned x = s_cnt[c][q];
                s_cnt[c][q] = run;
                run += x;
            }
        volatile unsigned long long* pub = scan.pub;
        unsigned long long prefix = 0;
        if (tile == 0) {
            pub[0] = kUFlagInclusive | run;
        } else {
            pub[tile] = kUFlagAggregate | run;
            long long t = tile - 1;
            unsigned long long t0 = 0;
            bool timed = false;
            while (t >= 0) {
                const unsigned long long v = pub[t];
                if ((v >> 62) == 0ull) {  // not published yet
                    if (!timed) {
                        t0 = u_globaltimer_ns();
                        timed = true;
                    } else if (u_globaltimer_ns() - t0 > scan.limit_ns) {
                        atomicExch(scan.status, kStatusTimeout);
                        break;
                    }
                    continue;
                }
                timed = false;
                prefix += v & kUCountMask;
                if ((v >> 62) == 2ull) break;
                --t;
            }
            pub[tile] = kUFlagInclusive | (prefix + run);
        }
        s_base = prefix;
        if (tile == (total - 1) / kUnionTile) *scan.total = prefix + run;
    }
    __syncthreads();
    const unsigned long long base = s_base;
#pragma unroll
    for (int c = 0; c < kUnionChunks; ++c) {
        if ((ball[c] >> lane) & 1u) {
            const long long s = tile * kUnionTile + c * 256 + tid;
            const unsigned long long pos = base + s_cnt[c][warp] + __popc(ball[c] & ((1u << lane) - 1u));
            mkey[pos] = ((unsigned long long)(s / k) << 32) | (unsigned long long)(unsigned)jv[c];
            mval[pos] = wv[c];
        }
    }
}

// The COO as (row << key_bits | col, weight) pairs for the radix sort
// (sort.cu), used below a size where the row-by-row build (coo.cu) pays.
// One thread per slot (i, t): union weight into w, and the COO pairs:
// (i, j) always, (j, i) too when i is absent from j's list (otherwise j's own
// slot emits it). Padding slots emit all-ones keys, which sort last.
__global__ void __launch_bounds__(256) union_pairs_kernel(const int32_t* __restrict__ idx,
                                                          const uint16_t* __restrict__ dist,
                                                          const WeightRow* __restrict__ rec, int n, int k,
                                                          float* __restrict__ w, int key_bits,
                                                          unsigned long long* __restrict__ keys,
                                                          float* __restrict__ vals, unsigned long long* nnz) {
    const long long total = (long long)n * k;
    unsigned long long local = 0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < total;
         s += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(s / k);
        const int j = idx[s];
        float wv = 0.0f;
        bool mutual = false;
        if (j >= 0) {
            const int d = dist[s];
            const WeightRow ri = rec[i];
            const WeightRow rj = rec[j];
            const float aij = umap_a(d, ri.rho, ri.sigma);
            mutual = in_list(rj, i, d);
            const float aji = mutual ? umap_a(d, rj.rho, rj.sigma) : 0.0f;
            wv = aij + aji - aij * aji;
        }
        w[s] = wv;
        if (keys) {
            const unsigned long long inval = ~0ull;
            if (j >= 0) {
                keys[2 * s] = ((unsigned long long)i << key_bits) | (unsigned long long)j;
                vals[2 * s] = wv;
                local += 1;
                if (!mutual) {
                    keys[2 * s + 1] = ((unsigned long long)j << key_bits) | (unsigned long long)i;
                    vals[2 * s + 1] = wv;
                    local += 1;
                } else {
                    keys[2 * s + 1] = inval;
                    vals[2 * s + 1] = 0.0f;
                }
            } else {
                keys[2 * s] = inval;
                keys[2 * s + 1] = inval;
                vals[2 * s] = 0.0f;
                vals[2 * s + 1] = 0.0f;
            }
        }
    }
    if (keys) {
        // warp then block aggregation of the valid-entry count
        for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(kFull, local, o);
        __shared__ unsigned long long s_cnt;
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        if ((threadIdx.x & 31) == 0 && local) atomicAdd(&s_cnt, local);
        __syncthreads();
        if (threadIdx.x == 0 && s_cnt) atomicAdd(nnz, s_cnt);
    }
}

__global__ void pairs_unpack_kernel(const unsigned long long* __restrict__ keys, const float* __restrict__ vals,
                                    int key_bits, const unsigned long long* __restrict__ nnz_dev, long long cap,
                                    int32_t* __restrict__ row, int32_t* __restrict__ col, float* __restrict__ w,
                                    int64_t* __restrict__ nnz_out) {
    const long long nnz = (long long)*nnz_dev;
    const unsigned long long mask = (1ull << key_bits) - 1ull;
    const long long lim = nnz < cap ? nnz : cap;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < lim;
         p += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[p];
        if (row) row[p] = (int32_t)(key >> key_bits);
        if (col) col[p] = (int32_t)(key & mask);
        if (w) w[p] = vals[p];
    }
    if (nnz_out && blockIdx.x == 0 && threadIdx.x == 0) *nnz_out = nnz;
}

int grid_for(long long work, int threads, int cap) {
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

size_t smooth_knn_smem_bytes(int32_t k) { return (size_t)kSkWarps * 32 * sk_stride(k) * sizeof(uint32_t); }

cudaError_t launch_smooth_knn(const int32_t* idx, const uint16_t* dist, int32_t n_rows, int32_t k, float T,
                              float* rho, float* sigma, WeightRow* rec, float* a, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    const size_t smem = smooth_knn_smem_bytes(k);
    if (smem > 48 * 1024) {
        static_assert(kSkWarps * 32 * 129 * 4 <= 227 * 1024, "staged rows of k = 256 fit a CTA");
        cudaError_t e = cudaFuncSetAttribute(smooth_knn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long long chunks = ((long long)n_rows + 31) / 32;
    const int grid = grid_for(chunks * 32, kSkThreads, device_sm_count() * 16);
    smooth_knn_kernel<<<grid, kSkThreads, smem, s>>>(idx, dist, n_rows, k, T, rho, sigma, rec, a);
    return cudaGetLastError();
}

cudaError_t launch_union(const int32_t* idx, const uint16_t* dist, const WeightRow* rec, int32_t n, int32_t k,
                         float* w, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = grid_for((long long)n * k, 256, device_sm_count() * 16);
    union_kernel<<<grid, 256, 0, s>>>(idx, dist, rec, n, k, w);
    return cudaGetLastError();
}

size_t union_scan_words(int32_t n, int32_t k) {
    return (size_t)(((long long)n * k + kUnionTile - 1) / kUnionTile);
}

cudaError_t launch_union_mirrors(const int32_t* idx, const uint16_t* dist, const WeightRow* rec, int32_t n,
                                 int32_t k, float* w, int32_t* kval, unsigned long long* mkey, float* mval,
                                 const UnionScan& scan, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long tiles = ((long long)n * k + kUnionTile - 1) / kUnionTile;
    union_mirrors_kernel<<<(unsigned)tiles, 256, 0, s>>>(idx, dist, rec, n, k, w, kval, mkey, mval, scan);
    return cudaGetLastError();
}

cudaError_t launch_union_pairs(const int32_t* idx, const uint16_t* dist, const WeightRow* rec, int32_t n, int32_t k,
                               float* w, int key_bits, unsigned long long* keys, float* vals, DeviceCounters* ctr,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = grid_for((long long)n * k, 256, device_sm_count() * 16);
    union_pairs_kernel<<<grid, 256, 0, s>>>(idx, dist, rec, n, k, w, key_bits, keys, vals,
                                            ctr ? &ctr->coo_nnz : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_pairs_unpack(const unsigned long long* keys, const float* vals, int key_bits,
                                const DeviceCounters* ctr, long long cap, int32_t* row, int32_t* col, float* w,
                                int64_t* nnz_out, cudaStream_t s) {
    const int grid = grid_for(cap > 0 ? cap : 1, 256, device_sm_count() * 16);
    pairs_unpack_kernel<<<grid, 256, 0, s>>>(keys, vals, key_bits, &ctr->coo_nnz, cap, row, col, w, nnz_out);
    return cudaGetLastError();
}

}  // namespace gumap
