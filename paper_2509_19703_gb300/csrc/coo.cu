// Symmetric COO of the fuzzy union, sorted by (row, col), built row by row.
//
// Row i of the union holds (i, j) for every j in i's kNN list (its own
// entries) and (i, j') for every j' whose list holds i while i's list does
// not hold j' (mirrors). A column never appears twice in a row: an own
// entry's column is in i's list, a mirror's is not. So the row is the merge
// of two sorted lists with distinct columns, i's own entries by column and
// its mirrors by id.
//
//   union_mirrors_kernel (weights.cu): the union weight of every slot, and
//     the mirrors compacted in slot order, keyed (source << 32) | target.
//   radix sort (sort.cu): a stable sort of the mirrors on the target's bits,
//     so each row's mirrors come out together and in ascending id (they
//     were in source order). No atomic counter is shared by the many rows
//     that list a hub, and no row needs sorting afterwards.
//   in_rows_kernel: each row's range [instart, inend) of sorted mirrors.
//   own_sort_kernel: one warp per row ranks its own entries by column.
//   row_scan_kernel: rowoff = exclusive prefix of the row lengths (own
//     entries plus mirrors) in one pass (decoupled look-back of Merrill and
//     Garland's single-pass scan).
//   own_emit_kernel: an own entry of rank r and column c lands at
//     rowoff + r + (the row's mirrors below c).
//   mirror_emit_kernel: the q-th mirror j' of row i lands at
//     rowoff + q + (own entries of row i below j').
// Every write lands inside its row: row lengths come from the counts, never
// from differences of rowoff, and rowoff never exceeds the true prefix (a
// look-back that gives up leaves it short and reports TIMEOUT).
#include "gumap_internal.cuh"

#include <climits>

namespace gumap {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                          // consecutive rows per thread
constexpr int kScanTile = kScanThreads * kScanItems;   // rows per tile
constexpr unsigned long long kFlagAggregate = 1ull << 62;  // this tile's sum only
constexpr unsigned long long kFlagInclusive = 2ull << 62;  // sum of this tile and all before it
constexpr unsigned long long kCountMask = (1ull << 62) - 1ull;
constexpr unsigned long long kLookbackLimitNs = 1000ull * 1000ull * 1000ull;
constexpr int kOwnThreads = 256;                       // own_sort_kernel: one warp per row

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ long long row_len(const CooArgs& a, long long i) {
    return (long long)a.kval[i] + (long long)a.mcnt[i];
}

__device__ __forceinline__ unsigned target_of(unsigned long long key, unsigned mask) { return (unsigned)key & mask; }

__device__ __forceinline__ long long mirror_count(const CooArgs& a) { return (long long)*a.mirrors; }

// Ranges of the sorted mirrors per target: a run of equal targets starts at
// instart and ends before inend.
__global__ void __launch_bounds__(256) in_rows_kernel(CooArgs a) {
    const unsigned mask = (1u << a.key_bits) - 1u;
    const long long count = mirror_count(a);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const unsigned t = target_of(a.tkey[p], mask);
        if (t >= (unsigned)a.n) continue;
        if (p == 0 || target_of(a.tkey[p - 1], mask) != t) a.instart[t] = (uint32_t)p;
        if (p == count - 1 || target_of(a.tkey[p + 1], mask) != t) a.inend[t] = (uint32_t)(p + 1);
    }
}

// One warp per row: the own entries (valid slots, distinct columns) ranked by
// column into scol / sw, and the row's mirror count. An entry's rank is the
// number of smaller columns in the row, counted against a shared-memory copy
// four columns per load.
__global__ void __launch_bounds__(kOwnThreads) own_sort_kernel(CooArgs a) {
    __shared__ __align__(16) int32_t s_col[kOwnThreads / 32][kMaxK];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int32_t* sc = s_col[wib];
    const int4* sv = reinterpret_cast<const int4*>(sc);
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int k = a.k;
    for (long long i = warp; i < a.n; i += nwarps) {
        const int kv = a.kval[i];
        const int kv4 = (kv + 3) & ~3;
        const size_t base = (size_t)i * k;
        for (int t = lane; t < kv4; t += 32) sc[t] = t < kv ? a.idx[base + t] : INT_MAX;  // columns are < INT_MAX
        __syncwarp();
        for (int t = lane; t < kv; t += 32) {
            const int x = sc[t];
            int r = 0;
            for (int f = 0; f < (kv4 >> 2); ++f) {
                const int4 v = sv[f];
                r += (v.x < x) + (v.y < x) + (v.z < x) + (v.w < x);
            }
            a.scol[base + r] = x;
            a.sw[base + r] = a.w[base + t];
        }
        if (lane == 0) a.mcnt[i] = a.inend[i] - a.instart[i];
        __syncwarp();  // s_col is rewritten by the next row
    }
}

__global__ void __launch_bounds__(kScanThreads) row_scan_kernel(CooArgs a) {
    __shared__ unsigned s_tile;
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&a.ctr[kCooCtrTile], 1u);
    __syncthreads();
    const long long tile = s_tile;
    const long long r0 = tile * kScanTile + (long long)tid * kScanItems;
    unsigned long long c[kScanItems];
    unsigned long long mine = 0;
#pragma unroll
    for (int e = 0; e < kScanItems; ++e) {
        const long long r = r0 + e;
        c[e] = r < a.n ? (unsigned long long)row_len(a, r) : 0ull;
        mine += c[e];
    }
    unsigned long long inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    unsigned long long wbase = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < warp) wbase += s_warp[w];
        total += s_warp[w];
    }
    if (tid == 0) {
        volatile unsigned long long* pub = a.pub;
        unsigned long long prefix = 0;
        if (tile == 0) {
            pub[0] = kFlagInclusive | total;
        } else {
            pub[tile] = kFlagAggregate | total;
            long long t = tile - 1;
            unsigned long long t0 = 0;
            bool timed = false;
            while (t >= 0) {
                const unsigned long long v = pub[t];
                if ((v >> 62) == 0ull) {  // not published yet
                    if (!timed) {
                        t0 = globaltimer_ns();
                        timed = true;
                    } else if (globaltimer_ns() - t0 > kLookbackLimitNs) {
                        atomicExch(a.status, kStatusTimeout);
                        break;
                    }
                    continue;
                }
                timed = false;
                prefix += v & kCountMask;
                if ((v >> 62) == 2ull) break;
                --t;
            }
            pub[tile] = kFlagInclusive | (prefix + total);
        }
        s_prefix = prefix;
        if (tile == (a.n - 1) / kScanTile) a.rowoff[a.n] = prefix + total;
    }
    __syncthreads();
    unsigned long long pos = s_prefix + wbase + inc - mine;
#pragma unroll
    for (int e = 0; e < kScanItems; ++e) {
        const long long r = r0 + e;
        if (r < a.n) a.rowoff[r] = pos;
        pos += c[e];
    }
}


// Number of mirrors of row i with an id below c: a binary search of the
// row's range of sorted mirrors (ids are the keys' high words).
__device__ __forceinline__ uint32_t in_below(const CooArgs& a, long long i, int c) {
    uint32_t lo = a.instart[i], hi = a.inend[i];
    const uint32_t first = lo;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((int)(a.tkey[mid] >> 32) < c) lo = mid + 1;
        else hi = mid;
    }
    return lo - first;
}

// One thread per slot: own entry of rank r (column c) of row i.
__global__ void __launch_bounds__(256) own_emit_kernel(CooArgs a) {
    const long long total = (long long)a.n * a.k;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < total;
         s += (long long)gridDim.x * blockDim.x) {
        const long long i = s / a.k;
        const int r = (int)(s - i * a.k);
        if (r >= a.kval[i]) continue;
        const int c = a.scol[s];
        const unsigned long long pos = a.rowoff[i] + (unsigned long long)r + in_below(a, i, c);
        a.ccol[pos] = c;
        a.cw[pos] = a.sw[s];
    }
}

// One thread per sorted mirror: the q-th mirror j' of row i.
__global__ void __launch_bounds__(256) mirror_emit_kernel(CooArgs a) {
    const unsigned mask = (1u << a.key_bits) - 1u;
    const long long count = mirror_count(a);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = a.tkey[p];
        const unsigned i = target_of(key, mask);
        const int src = (int)(key >> 32);
        const size_t base = (size_t)i * a.k;
        int lo = 0, hi = a.kval[i];  // own entries of row i with a column below src
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a.scol[base + mid] < src) lo = mid + 1;
            else hi = mid;
        }
        const unsigned long long q = (unsigned long long)(p - a.instart[i]);
        const unsigned long long pos = a.rowoff[i] + q + (unsigned long long)lo;
        a.ccol[pos] = src;
        a.cw[pos] = a.tval[p];
    }
}

__global__ void __launch_bounds__(256) coo_unpack_kernel(CooArgs a, long long cap, int32_t* __restrict__ row,
                                                         int32_t* __restrict__ col, float* __restrict__ w,
                                                         int64_t* __restrict__ nnz_out) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < a.n; i += nwarps) {
        const unsigned long long base = a.rowoff[i];
        const long long c = row_len(a, i);
        for (long long e = lane; e < c; e += 32) {
            const unsigned long long p = base + e;
            if (p >= (unsigned long long)cap) break;
            if (row) row[p] = (int32_t)i;
            if (col) col[p] = a.ccol[p];
            if (w) w[p] = a.cw[p];
        }
    }
    if (nnz_out && blockIdx.x == 0 && threadIdx.x == 0) *nnz_out = (int64_t)a.rowoff[a.n];
}

int grid_for(long long work, int threads, int cap) {
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

size_t pad16(size_t b) { return (b + 15) & ~(size_t)15; }

}  // namespace

size_t coo_scratch_bytes(int32_t n) {
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const size_t tiles = (nn + kScanTile - 1) / kScanTile;
    return 2 * pad16(nn * sizeof(uint32_t)) + pad16(kCooCtrWords * sizeof(uint32_t)) +
           tiles * sizeof(unsigned long long);
}

void coo_scratch_split(void* scratch, int32_t n, uint32_t** instart, uint32_t** inend, uint32_t** ctr,
                       unsigned long long** pub) {
    const size_t m = pad16((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
    char* p = static_cast<char*>(scratch);
    *instart = reinterpret_cast<uint32_t*>(p);
    *inend = reinterpret_cast<uint32_t*>(p + m);
    *ctr = reinterpret_cast<uint32_t*>(p + 2 * m);
    *pub = reinterpret_cast<unsigned long long*>(p + 2 * m + pad16(kCooCtrWords * sizeof(uint32_t)));
}

cudaError_t launch_coo_build(const CooArgs& a, int sms, cudaStream_t s, int* launches) {
    if (a.n <= 0) return cudaSuccess;
    const long long slots = (long long)a.n * a.k;
    in_rows_kernel<<<grid_for(slots, 256, sms * 16), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    own_sort_kernel<<<grid_for((long long)a.n * 32, kOwnThreads, sms * 8), kOwnThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long tiles = ((long long)a.n + kScanTile - 1) / kScanTile;
    row_scan_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    own_emit_kernel<<<grid_for(slots, 256, sms * 16), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mirror_emit_kernel<<<grid_for(slots, 256, sms * 16), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (launches) *launches += 5;
    return cudaSuccess;
}

cudaError_t launch_coo_unpack(const CooArgs& a, long long cap, int32_t* row, int32_t* col, float* w,
                              int64_t* nnz_out, cudaStream_t s) {
    const int grid = grid_for((long long)(a.n > 0 ? a.n : 1) * 32, 256, device_sm_count() * 16);
    coo_unpack_kernel<<<grid, 256, 0, s>>>(a, cap, row, col, w, nnz_out);
    return cudaGetLastError();
}

}  // namespace gumap
