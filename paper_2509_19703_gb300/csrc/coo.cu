// Symmetric COO of the fuzzy union, sorted by (row, col), built row by row.
//
// Row i of the union holds (i, j) for every j in i's kNN list (its own
// entries) and (i, j') for every j' whose list holds i while i's list does
// not hold j' (mirrors). A column never appears twice in a row: an own
// entry's column is in i's list, a mirror's is not. So every row is a set
// of distinct columns and its order by column is unique.
//
//   union_kernel (weights.cu): the union weight of every slot; per row the
//     number of own entries kval[i] and of mirrors mcnt[j] (an atomic whose
//     old value is the mirror's rank mpos within its row).
//   row_scan_kernel: rowoff = exclusive prefix of kval + mcnt over the rows
//     in one pass (decoupled look-back of Merrill and Garland's single-pass
//     scan); rows longer than kWarpRow go on a list.
//   scatter_kernel: own entry (i, t) to rowoff[i] + t, mirror to rowoff[j] +
//     kval[j] + mpos (column and weight; unordered within the row).
//   row_sort_warp_kernel: rows of up to kWarpRow entries, one warp each; the
//     place of an entry is the number of smaller columns in its row, counted
//     against the row's columns in shared memory.
//   row_sort_large_kernel: longer rows, one CTA each; a bitmap of the row's
//     column range in shared memory (2^19 columns per chunk) whose popcount
//     prefix is the place of each column.
// Every write lands inside [0, 2 n k): row lengths are taken from kval +
// mcnt, never from differences of rowoff, and rowoff never exceeds the true
// prefix (a look-back that gives up leaves it short and reports TIMEOUT).
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
constexpr int kSortThreads = 256;
constexpr int kWarpRow = 1024;                         // longest row sorted by one warp
constexpr int kLargeThreads = 512;
constexpr int kChunkWords = 16384;                     // bitmap words per chunk: 2^19 columns
constexpr int kWordsPerWarp = kChunkWords / (kLargeThreads / 32);
constexpr long long kChunkCols = 32ll * kChunkWords;
constexpr size_t kLargeSmem = 2 * kChunkWords * sizeof(uint32_t);  // bitmap + word prefix: 128 KB

static_assert(kWordsPerWarp % 32 == 0 && kWordsPerWarp * (kLargeThreads / 32) == kChunkWords, "chunk words per warp");
static_assert(kWarpRow % 4 == 0, "shared rows hold whole int4 groups");

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ long long row_len(const CooArgs& a, long long i) {
    return (long long)a.kval[i] + (long long)a.mcnt[i];
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
        if (r < a.n && c[e] > (unsigned long long)kWarpRow) a.large[atomicAdd(&a.ctr[kCooCtrLarge], 1u)] = (int32_t)r;
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

__global__ void __launch_bounds__(256) scatter_kernel(CooArgs a) {
    const long long total = (long long)a.n * a.k;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < total;
         s += (long long)gridDim.x * blockDim.x) {
        const int j = a.idx[s];
        if (j < 0) continue;
        const long long i = s / a.k;
        const long long t = s - i * a.k;
        const float wv = a.w[s];
        const unsigned long long po = a.rowoff[i] + (unsigned long long)t;
        a.tcol[po] = j;
        a.tw[po] = wv;
        const uint32_t m = a.mpos[s];
        if (m != kNoMirror) {
            const unsigned long long pm = a.rowoff[j] + (unsigned long long)a.kval[j] + m;
            a.tcol[pm] = (int32_t)i;
            a.tw[pm] = wv;
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) row_sort_warp_kernel(CooArgs a) {
    __shared__ __align__(16) int32_t s_col[kSortThreads / 32][kWarpRow];
    const int lane = threadIdx.x & 31;
    int32_t* sc = s_col[threadIdx.x >> 5];
    const int4* sv = reinterpret_cast<const int4*>(sc);
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < a.n; i += nwarps) {
        const int c = (int)min(row_len(a, i), (long long)kWarpRow + 1);
        if (c == 0 || c > kWarpRow) continue;  // empty, or a long row (row_sort_large_kernel)
        const unsigned long long base = a.rowoff[i];
        const int c4 = (c + 3) & ~3;
        for (int e = lane; e < c4; e += 32) sc[e] = e < c ? a.tcol[base + e] : INT_MAX;  // columns are < INT_MAX
        __syncwarp();
        for (int e0 = lane; e0 < c; e0 += 64) {
            const int e1 = e0 + 32;
            const int x0 = sc[e0];
            const int x1 = e1 < c ? sc[e1] : INT_MAX;
            int r0 = 0, r1 = 0;
            for (int f = 0; f < (c4 >> 2); ++f) {
                const int4 v = sv[f];
                r0 += (v.x < x0) + (v.y < x0) + (v.z < x0) + (v.w < x0);
                r1 += (v.x < x1) + (v.y < x1) + (v.z < x1) + (v.w < x1);
            }
            a.ccol[base + r0] = x0;
            a.cw[base + r0] = a.tw[base + e0];
            if (e1 < c) {
                a.ccol[base + r1] = x1;
                a.cw[base + r1] = a.tw[base + e1];
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kLargeThreads) row_sort_large_kernel(CooArgs a) {
    extern __shared__ uint32_t sm[];
    uint32_t* bm = sm;                 // bitmap of the chunk's columns
    uint32_t* pre = sm + kChunkWords;  // per word: set bits in the chunk's words before it
    __shared__ int s_row, s_lo, s_hi;
    __shared__ unsigned s_warp[kLargeThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned nlarge = a.ctr[kCooCtrLarge];
    for (;;) {
        if (tid == 0) {
            const unsigned r = atomicAdd(&a.ctr[kCooCtrNextLarge], 1u);
            s_row = r < nlarge ? a.large[r] : -1;
            s_lo = INT_MAX;
            s_hi = -1;
        }
        __syncthreads();
        const int i = s_row;
        if (i < 0) break;
        const long long c = row_len(a, i);
        const unsigned long long base = a.rowoff[i];
        int lo = INT_MAX, hi = -1;
        for (long long e = tid; e < c; e += kLargeThreads) {
            const int x = a.tcol[base + e];
            lo = min(lo, x);
            hi = max(hi, x);
        }
        lo = __reduce_min_sync(kFull, lo);
        hi = __reduce_max_sync(kFull, hi);
        if (lane == 0) {
            atomicMin(&s_lo, lo);
            atomicMax(&s_hi, hi);
        }
        __syncthreads();
        const long long row_lo = s_lo, row_hi = s_hi;
        unsigned long long run = 0;  // columns of the row in earlier chunks
        for (long long cb = row_lo; cb <= row_hi; cb += kChunkCols) {
            for (int wi = tid; wi < kChunkWords; wi += kLargeThreads) bm[wi] = 0u;
            __syncthreads();
            for (long long e = tid; e < c; e += kLargeThreads) {
                const long long off = (long long)a.tcol[base + e] - cb;
                if (off >= 0 && off < kChunkCols) atomicOr(&bm[off >> 5], 1u << (off & 31));
            }
            __syncthreads();
            // exclusive prefix of the words' popcounts: warp w owns words
            // [w * kWordsPerWarp, (w + 1) * kWordsPerWarp), read 32 at a time
            // (one per lane, no bank conflict)
            const int wb = warp * kWordsPerWarp;
            unsigned mine = 0;
            for (int q = 0; q < kWordsPerWarp / 32; ++q) mine += __popc(bm[wb + q * 32 + lane]);
            mine = __reduce_add_sync(kFull, mine);
            if (lane == 0) s_warp[warp] = mine;
            __syncthreads();
            unsigned carry = 0, chunk_total = 0;
#pragma unroll
            for (int w = 0; w < kLargeThreads / 32; ++w) {
                if (w < warp) carry += s_warp[w];
                chunk_total += s_warp[w];
            }
            for (int q = 0; q < kWordsPerWarp / 32; ++q) {
                const unsigned pc = __popc(bm[wb + q * 32 + lane]);
                unsigned inc = pc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(kFull, inc, o);
                    if (lane >= o) inc += y;
                }
                pre[wb + q * 32 + lane] = carry + inc - pc;
                carry += __shfl_sync(kFull, inc, 31);
            }
            __syncthreads();
            for (long long e = tid; e < c; e += kLargeThreads) {
                const int x = a.tcol[base + e];
                const long long off = (long long)x - cb;
                if (off >= 0 && off < kChunkCols) {
                    const int wi = (int)(off >> 5);
                    const unsigned r = pre[wi] + __popc(bm[wi] & ((1u << (off & 31)) - 1u));
                    const unsigned long long pos = base + run + r;
                    a.ccol[pos] = x;
                    a.cw[pos] = a.tw[base + e];
                }
            }
            run += chunk_total;
            __syncthreads();  // s_warp, bm and pre are rewritten by the next chunk
        }
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

}  // namespace

size_t coo_scratch_bytes(int32_t n) {
    const size_t tiles = (size_t)((n > 0 ? n : 1) + kScanTile - 1) / kScanTile;
    const size_t mcnt = ((size_t)(n > 0 ? n : 1) * sizeof(uint32_t) + 15) & ~(size_t)15;
    return mcnt + kCooCtrWords * sizeof(uint32_t) + tiles * sizeof(unsigned long long);
}

void coo_scratch_split(void* scratch, int32_t n, uint32_t** mcnt, uint32_t** ctr, unsigned long long** pub) {
    const size_t m = ((size_t)(n > 0 ? n : 1) * sizeof(uint32_t) + 15) & ~(size_t)15;
    char* p = static_cast<char*>(scratch);
    *mcnt = reinterpret_cast<uint32_t*>(p);
    *ctr = reinterpret_cast<uint32_t*>(p + m);
    *pub = reinterpret_cast<unsigned long long*>(p + m + kCooCtrWords * sizeof(uint32_t));
}

cudaError_t launch_coo_build(const CooArgs& a, int sms, cudaStream_t s, int* launches) {
    if (a.n <= 0) return cudaSuccess;
    const long long tiles = ((long long)a.n + kScanTile - 1) / kScanTile;
    row_scan_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scatter_kernel<<<grid_for((long long)a.n * a.k, 256, sms * 16), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    row_sort_warp_kernel<<<grid_for((long long)a.n * 32, kSortThreads, sms * 8), kSortThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(row_sort_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kLargeSmem)) != cudaSuccess)
        return e;
    row_sort_large_kernel<<<sms, kLargeThreads, kLargeSmem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (launches) *launches += 4;
    return cudaSuccess;
}

cudaError_t launch_coo_unpack(const CooArgs& a, long long cap, int32_t* row, int32_t* col, float* w,
                              int64_t* nnz_out, cudaStream_t s) {
    const int grid = grid_for((long long)(a.n > 0 ? a.n : 1) * 32, 256, device_sm_count() * 16);
    coo_unpack_kernel<<<grid, 256, 0, s>>>(a, cap, row, col, w, nnz_out);
    return cudaGetLastError();
}

}  // namespace gumap
