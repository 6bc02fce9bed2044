// UMAP fuzzy weights of the kNN lists (Section 2.1, h_ij) and their fuzzy
// union (the symmetrisation of the UMAP implementation the paper builds on,
// Section 4.1.1).
//
// smooth_knn: one warp per row. rho_i is the smallest valid distance of the
// row; sigma_i solves f(sigma) = sum_j exp(-max(0, d_ij - rho_i)/sigma) = T
// with T = log2 k, by FP32 bisection on a bracket [0, hi] whose hi doubles
// until f(hi) >= T. f rises strictly from c_eq = #{j : d_ij = rho_i} (sigma
// -> 0) to kv = #valid (sigma -> inf), so a root exists iff c_eq < T < kv:
//   kv <= T   -> no root, sigma = +inf, every weight 1;
//   c_eq >= T -> no root, sigma -> 0+, lifted by the floor;
// and sigma = max(sigma*, 1e-3 * mean_j d_ij). Both decisions compare exact
// integers with T, and log2 k is at least 0.0056 away from any integer for a
// k that is not a power of two, so FP32 and FP64 take the same branch.
//
// union: w_ij = a_ij + a_ji - a_ij a_ji with a_ji = 0 when i is not in j's
// list. Hop distances are symmetric, so i can sit in j's list only at
// distance d_ij; the lookup binary-searches the run of row j with that
// distance (rows are sorted by (distance, id)).
#include "gumap_internal.cuh"

#include <math_constants.h>

namespace gumap {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// f(sigma) for the lane's slots, summed over the warp (every lane gets the
// bitwise-identical total, so all lanes take the same bisection branch).
__device__ __forceinline__ float f_sigma(const int (&dl)[kMaxK / 32], int rho, float sigma) {
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < kMaxK / 32; ++q) {
        if (dl[q] >= 0) acc += expf(-(float)(dl[q] - rho) / sigma);
    }
    return warp_sum(acc);
}

__global__ void __launch_bounds__(256) smooth_knn_kernel(const uint16_t* __restrict__ dist, int n_rows, int k,
                                                         float T, float* __restrict__ rho_out,
                                                         float* __restrict__ sigma_out, float* __restrict__ a_out) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int nloc = (k + 31) >> 5;  // slots per lane (<= 8)
    for (long long i = warp; i < n_rows; i += nwarps) {
        const uint16_t* d = dist + (size_t)i * k;
        int dl[kMaxK / 32];
        int kv = 0, dmin = 0x7FFFFFFF;
        long long sum = 0;
#pragma unroll
        for (int q = 0; q < kMaxK / 32; ++q) {
            dl[q] = -1;
            const int t = lane + 32 * q;
            if (q < nloc && t < k) {
                const int x = d[t];
                if (x != kDistInf) {
                    dl[q] = x;
                    kv++;
                    sum += x;
                    dmin = min(dmin, x);
                }
            }
        }
        kv = __reduce_add_sync(kFull, kv);
        float* arow = a_out + (size_t)i * k;
        if (kv == 0) {
            for (int t = lane; t < k; t += 32) arow[t] = 0.0f;
            if (lane == 0) {
                rho_out[i] = 0.0f;
                sigma_out[i] = 0.0f;
            }
            continue;
        }
        const int rho = __reduce_min_sync(kFull, dmin);
        int ceq = 0;
#pragma unroll
        for (int q = 0; q < kMaxK / 32; ++q) ceq += (dl[q] == rho) ? 1 : 0;
        ceq = __reduce_add_sync(kFull, ceq);
        // sum of at most 256 uint16 values fits in int32
        const int isum = __reduce_add_sync(kFull, (int)sum);
        const float mean = (float)isum / (float)kv;
        float sigma;
        if ((float)kv <= T) {
            sigma = CUDART_INF_F;
        } else if ((float)ceq >= T) {
            sigma = 0.0f;
        } else {
            float lo = 0.0f, hi = 1.0f;
            for (int it = 0; it < 128 && f_sigma(dl, rho, hi) < T; ++it) hi *= 2.0f;
            for (int it = 0; it < 200; ++it) {
                const float mid = 0.5f * (lo + hi);
                if (!(mid > lo && mid < hi)) break;
                if (f_sigma(dl, rho, mid) > T) hi = mid;
                else lo = mid;
            }
            sigma = 0.5f * (lo + hi);
        }
        sigma = fmaxf(sigma, 1e-3f * mean);
#pragma unroll
        for (int q = 0; q < kMaxK / 32; ++q) {
            const int t = lane + 32 * q;
            if (q < nloc && t < k) {
                float v = 0.0f;
                if (dl[q] >= 0) v = isinf(sigma) ? 1.0f : expf(-(float)(dl[q] - rho) / sigma);
                arow[t] = v;
            }
        }
        if (lane == 0) {
            rho_out[i] = (float)rho;
            sigma_out[i] = sigma;
        }
    }
}

// Position of i in row j of the lists, or -1. The row is sorted by
// (distance, id); i can only appear at distance dij.
__device__ __forceinline__ int find_in_row(const int32_t* __restrict__ idx, const uint16_t* __restrict__ dist,
                                           int k, int j, int i, int dij) {
    const int32_t* ri = idx + (size_t)j * k;
    const uint16_t* rd = dist + (size_t)j * k;
    // lower bound of (dij, i) in the (distance, id) order; padding sorts last
    int lo = 0, hi = k;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int dm = rd[mid];
        const int im = ri[mid];
        const bool less = (dm < dij) || (dm == dij && im < i);
        if (less && dm != kDistInf) lo = mid + 1;
        else hi = mid;
    }
    return (lo < k && rd[lo] == dij && ri[lo] == i) ? lo : -1;
}

// One thread per slot (i, t): union weight into w. With mcnt given, also
// what the row-by-row COO build needs (coo.cu): a slot whose target j does
// not list i is a mirror in row j and takes the next place among j's
// mirrors (mpos; kNoMirror otherwise), and the row's own entries are its
// valid slots, which come first (kval).
__global__ void __launch_bounds__(256) union_kernel(const int32_t* __restrict__ idx,
                                                    const uint16_t* __restrict__ dist,
                                                    const float* __restrict__ a, int n, int k,
                                                    float* __restrict__ w, uint32_t* __restrict__ mcnt,
                                                    uint32_t* __restrict__ mpos, int32_t* __restrict__ kval) {
    const long long total = (long long)n * k;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < total;
         s += (long long)gridDim.x * blockDim.x) {
        const long long i = s / k;
        const int t = (int)(s - i * k);
        const int j = idx[s];
        float wv = 0.0f;
        bool mutual = false;
        if (j >= 0) {
            const float aij = a[s];
            const int p = find_in_row(idx, dist, k, j, (int)i, dist[s]);
            const float aji = p >= 0 ? a[(size_t)j * k + p] : 0.0f;
            mutual = p >= 0;
            wv = aij + aji - aij * aji;
        }
        w[s] = wv;
        if (mcnt) {
            if (j >= 0) {
                mpos[s] = mutual ? kNoMirror : atomicAdd(&mcnt[j], 1u);
                if (t == k - 1 || idx[s + 1] < 0) kval[i] = t + 1;
            } else {
                mpos[s] = kNoMirror;
                if (t == 0) kval[i] = 0;
            }
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
                                                    const float* __restrict__ a, int n, int k,
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
            const float aij = a[s];
            const int p = find_in_row(idx, dist, k, j, i, dist[s]);
            const float aji = p >= 0 ? a[(size_t)j * k + p] : 0.0f;
            mutual = p >= 0;
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

cudaError_t launch_smooth_knn(const uint16_t* dist, int32_t n_rows, int32_t k, float T, float* rho, float* sigma,
                              float* a, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    const int grid = grid_for((long long)n_rows * 32, 256, 152 * 16);
    smooth_knn_kernel<<<grid, 256, 0, s>>>(dist, n_rows, k, T, rho, sigma, a);
    return cudaGetLastError();
}

cudaError_t launch_union(const int32_t* idx, const uint16_t* dist, const float* a, int32_t n, int32_t k, float* w,
                         uint32_t* mcnt, uint32_t* mpos, int32_t* kval, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = grid_for((long long)n * k, 256, 152 * 16);
    union_kernel<<<grid, 256, 0, s>>>(idx, dist, a, n, k, w, mcnt, mpos, kval);
    return cudaGetLastError();
}

cudaError_t launch_union_pairs(const int32_t* idx, const uint16_t* dist, const float* a, int32_t n, int32_t k,
                               float* w, int key_bits, unsigned long long* keys, float* vals, DeviceCounters* ctr,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = grid_for((long long)n * k, 256, 152 * 16);
    union_pairs_kernel<<<grid, 256, 0, s>>>(idx, dist, a, n, k, w, key_bits, keys, vals, ctr ? &ctr->coo_nnz : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_pairs_unpack(const unsigned long long* keys, const float* vals, int key_bits,
                                const DeviceCounters* ctr, long long cap, int32_t* row, int32_t* col, float* w,
                                int64_t* nnz_out, cudaStream_t s) {
    const int grid = grid_for(cap > 0 ? cap : 1, 256, 152 * 16);
    pairs_unpack_kernel<<<grid, 256, 0, s>>>(keys, vals, key_bits, &ctr->coo_nnz, cap, row, col, w, nnz_out);
    return cudaGetLastError();
}

}  // namespace gumap
