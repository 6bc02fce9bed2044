// LSD radix sort of (uint64 key, float value) pairs on the low `bits` key
// bits, 8 bits per pass. Used to order the fuzzy-union COO by (row, col):
// the key of entry (i, j) is (i << B) | j with B = ceil(log2 n).
//
// Each pass: (1) a tile histogram of the digit (256 bins per 4096-key tile,
// stored digit-major), (2) one CTA per digit scans that digit's tile counts
// and records the digit total, (3) a stable scatter: each tile adds the
// prefix of the digit totals to its tile offsets, then ranks its keys in
// input order with warp match/ballot ranks plus per-warp digit counts in
// shared memory.
#include "gumap_internal.cuh"

namespace gumap {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

__global__ void __launch_bounds__(kThreads) hist_kernel(const unsigned long long* __restrict__ keys,
                                                        long long count, int shift, int num_tiles,
                                                        unsigned int* __restrict__ hist) {
    __shared__ unsigned int h[256];
    const int tid = threadIdx.x;
    h[tid] = 0u;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kTile;
    unsigned int dg[kItems];
#pragma unroll
    for (int c = 0; c < kItems; ++c) {  // all loads in flight before the counting
        const long long i = base + c * kThreads + tid;
        dg[c] = i < count ? (unsigned)(__ldcs(keys + i) >> shift) & 0xFFu : 256u;
    }
#pragma unroll
    for (int c = 0; c < kItems; ++c)
        if (dg[c] < 256u) atomicAdd(&h[dg[c]], 1u);
    __syncthreads();
    hist[(size_t)tid * num_tiles + blockIdx.x] = h[tid];
}

// One CTA per digit: exclusive scan, in place, of that digit's per-tile
// counts (the tile offsets within the digit's output range), and the digit's
// total into totals[digit]. 4096 entries per round: each thread scans 4
// consecutive entries, warps scan with shuffles, warp totals are scanned by
// warp 0, a running carry links the rounds. Every load is coalesced.
__global__ void __launch_bounds__(1024) scan_kernel(unsigned int* __restrict__ hist, long long len,
                                                    unsigned int* __restrict__ totals) {
    __shared__ unsigned int wsum[32];
    __shared__ unsigned int carry_s;
    unsigned int* data = hist + (size_t)blockIdx.x * len;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry_s = 0u;
    __syncthreads();
    for (long long base = 0; base < len; base += 4096) {
        const long long i0 = base + 4ll * tid;
        unsigned int x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = (i0 + q < len) ? data[i0 + q] : 0u;
        const unsigned int t = x[0] + x[1] + x[2] + x[3];
        unsigned int inc = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            unsigned int w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(kFull, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const unsigned int carry = carry_s;
        unsigned int run = carry + (warp > 0 ? wsum[warp - 1] : 0u) + (inc - t);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (i0 + q < len) data[i0 + q] = run;
            run += x[q];
        }
        __syncthreads();
        if (tid == 0) carry_s = carry + wsum[31];
        __syncthreads();
    }
    if (tid == 0) totals[blockIdx.x] = carry_s;
}

__global__ void __launch_bounds__(kThreads) scatter_kernel(const unsigned long long* __restrict__ kin,
                                                           const float* __restrict__ vin,
                                                           unsigned long long* __restrict__ kout,
                                                           float* __restrict__ vout, long long count, int shift,
                                                           int num_tiles, const unsigned int* __restrict__ offs,
                                                           const unsigned int* __restrict__ totals) {
    __shared__ unsigned int run[256];
    __shared__ unsigned int wcnt[kWarps][256];
    __shared__ unsigned int wtot[kWarps];
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    // start of digit tid's output range: exclusive prefix of the digit totals
    const unsigned int tot = totals[tid];
    unsigned int inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wtot[warp] = inc;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0u;
    __syncthreads();
    unsigned int before = inc - tot;
    for (int w = 0; w < warp; ++w) before += wtot[w];
    run[tid] = before + offs[(size_t)tid * num_tiles + blockIdx.x];
    __syncthreads();
    const long long base = (long long)blockIdx.x * kTile;
    // the tile's keys and values are loaded up front: one memory latency, not 16
    unsigned long long keys[kItems];
    float vals[kItems];
#pragma unroll
    for (int c = 0; c < kItems; ++c) {
        const long long i = base + c * kThreads + tid;
        keys[c] = i < count ? __ldcs(kin + i) : 0ull;
        vals[c] = i < count ? __ldcs(vin + i) : 0.0f;
    }
#pragma unroll
    for (int c = 0; c < kItems; ++c) {
        const long long i = base + c * kThreads + tid;
        const bool valid = i < count;
        const unsigned long long key = keys[c];
        const float val = vals[c];
        const int d = valid ? (int)((key >> shift) & 0xFFull) : 256;  // invalid lanes group apart
        const unsigned peers = __match_any_sync(kFull, d);
        const unsigned rank = __popc(peers & lt);
        if (valid && rank == 0u) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned int pos = run[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        unsigned int tot = 0u;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            tot += wcnt[w][tid];
            wcnt[w][tid] = 0u;
        }
        run[tid] += tot;
        __syncthreads();
    }
}

}  // namespace

size_t radix_sort_temp_bytes(long long count) {
    const long long tiles = (count + kTile - 1) / kTile;
    return (size_t)(256 * (tiles > 0 ? tiles : 1) + 256) * sizeof(unsigned int);  // + digit totals
}

cudaError_t radix_sort_pairs(unsigned long long* keys, float* vals, unsigned long long* keys_tmp, float* vals_tmp,
                             long long count, int bits, void* temp, size_t temp_bytes, cudaStream_t s,
                             unsigned long long** keys_out, float** vals_out, int* launches) {
    *keys_out = keys;
    *vals_out = vals;
    if (count <= 1 || bits <= 0) return cudaSuccess;
    if (count > 0xFFFFFFFFll) return cudaErrorInvalidValue;  // 32-bit output offsets
    const long long tiles = (count + kTile - 1) / kTile;
    if (temp_bytes < radix_sort_temp_bytes(count)) return cudaErrorInvalidValue;
    unsigned int* hist = static_cast<unsigned int*>(temp);
    unsigned int* totals = hist + 256 * tiles;
    unsigned long long *ka = keys, *kb = keys_tmp;
    float *va = vals, *vb = vals_tmp;
    for (int shift = 0; shift < bits; shift += 8) {
        hist_kernel<<<(unsigned)tiles, kThreads, 0, s>>>(ka, count, shift, (int)tiles, hist);
        scan_kernel<<<256, 1024, 0, s>>>(hist, tiles, totals);
        scatter_kernel<<<(unsigned)tiles, kThreads, 0, s>>>(ka, va, kb, vb, count, shift, (int)tiles, hist, totals);
        if (launches) *launches += 3;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        unsigned long long* tk = ka;
        ka = kb;
        kb = tk;
        float* tv = va;
        va = vb;
        vb = tv;
    }
    *keys_out = ka;
    *vals_out = va;
    return cudaSuccess;
}

}  // namespace gumap
