// LSD radix sort of (uint64 key, float value) pairs on the low `bits` key
// bits, 8 bits per pass. Used to order the fuzzy-union COO by (row, col):
// the key of entry (i, j) is (i << B) | j with B = ceil(log2 n).
//
// One-sweep organisation (the decoupled look-back of Merrill and Garland's
// single-pass scan, applied per digit as in Adinets and Merrill's Onesweep
// radix sort): one kernel counts the digits of every pass in a single read
// of the keys; then one kernel per pass, in which each CTA takes the next
// tile id from a counter, ranks its 4096 keys by digit (stable: warp w owns
// the w-th 512-key segment of the tile, ranked with warp match), publishes
// its per-digit counts, adds the counts of the tiles before it by looking
// back over their published words, lays the tile out in shared memory in
// digit order and writes it from there, so consecutive threads store
// consecutive elements of each digit's run. A tile only waits on tiles with
// smaller ids, which were handed out earlier to CTAs already running, so the
// waits end; each is bounded in time all the same and reports
// GUMAP_ERR_TIMEOUT in the caller's status word when it gives up. The sort
// is stable, which the transpose of the union COO relies on.
#include "gumap_internal.cuh"

namespace gumap {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                     // keys per lane
constexpr int kTile = kThreads * kItems;       // 4096 keys per tile
constexpr int kSeg = 32 * kItems;              // keys of one warp's segment
constexpr size_t kStageBytes = (size_t)kTile * (sizeof(unsigned long long) + sizeof(float));
constexpr int kMaxPasses = 8;
constexpr unsigned kFull = 0xFFFFFFFFu;
// published word of (tile, digit): flag in the top two bits, count below
constexpr unsigned long long kFlagAggregate = 1ull << 62;  // this tile's count only
constexpr unsigned long long kFlagInclusive = 2ull << 62;  // count of this tile and all before it
constexpr unsigned long long kCountMask = (1ull << 62) - 1ull;
constexpr unsigned long long kLookbackLimitNs = 1000ull * 1000ull * 1000ull;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Counts of every digit of every pass, one read of the keys: hist[p][d].
// The element count: `count`, or the device count when one is given (at most `count`).
__device__ __forceinline__ long long live_count(long long count, const unsigned long long* count_dev) {
    if (!count_dev) return count;
    const unsigned long long c = *count_dev;
    return c < (unsigned long long)count ? (long long)c : count;
}

__global__ void __launch_bounds__(kThreads) hist_all_kernel(const unsigned long long* __restrict__ keys,
                                                            long long count, int passes,
                                                            unsigned int* __restrict__ hist,
                                                            const unsigned long long* count_dev) {
    __shared__ unsigned int h[kMaxPasses][256];
    count = live_count(count, count_dev);
    for (int p = 0; p < passes; ++p) h[p][threadIdx.x] = 0u;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = __ldg(keys + i);
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(unsigned)(k >> (8 * p)) & 0xFFu], 1u);
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p)
        if (h[p][threadIdx.x]) atomicAdd(&hist[p * 256 + threadIdx.x], h[p][threadIdx.x]);
}

// One pass (digit at bit `shift`). hist: this pass's digit counts; tile_ctr:
// this pass's tile counter; pub: this pass's published words [tiles][256];
// all zeroed before the first pass. Dynamic shared memory: the tile's keys
// and values in digit order (kStageBytes).
__global__ void __launch_bounds__(kThreads, 2) onesweep_kernel(const unsigned long long* __restrict__ kin,
                                                               const float* __restrict__ vin,
                                                               unsigned long long* __restrict__ kout,
                                                               float* __restrict__ vout, long long count, int shift,
                                                               const unsigned int* __restrict__ hist,
                                                               unsigned int* tile_ctr, unsigned long long* pub,
                                                               int32_t* status, const unsigned long long* count_dev) {
    extern __shared__ __align__(16) unsigned char os_smem[];
    unsigned long long* skey = reinterpret_cast<unsigned long long*>(os_smem);
    float* sval = reinterpret_cast<float*>(skey + kTile);
    __shared__ unsigned int s_tile;
    __shared__ unsigned int wcnt[kWarps][256];  // per-warp digit counts, then per-warp offsets in the digit's run
    __shared__ unsigned int tstart[256];        // the digit's first place in the tile's digit order
    __shared__ long long gshift[256];           // global place of the tile's digit-d run, minus tstart[d]
    __shared__ unsigned int wsum[kWarps];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0u;
    __syncthreads();
    const long long tile = s_tile;
    count = live_count(count, count_dev);
    // tiles past the live count take no part: only later tiles would look back at them
    if (tile * kTile >= count && tile > 0) return;
    const long long seg = tile * kTile + (long long)warp * kSeg;

    // load the warp's segment (coalesced), then rank it: rank[c] is the
    // key's position among the segment's keys of the same digit
    unsigned long long key[kItems];
    float val[kItems];
    unsigned int rank[kItems];
    // digit of item c, or 256 past the end (invalid keys rank apart)
    auto digit = [&](int c) -> int {
        return seg + c * 32 + lane < count ? (int)((key[c] >> shift) & 0xFFull) : 256;
    };
#pragma unroll
    for (int c = 0; c < kItems; ++c) {
        const long long i = seg + c * 32 + lane;
        key[c] = i < count ? __ldcs(kin + i) : 0ull;
        val[c] = i < count ? __ldcs(vin + i) : 0.0f;
    }
#pragma unroll
    for (int c = 0; c < kItems; ++c) {
        const int d = digit(c);
        const unsigned peers = __match_any_sync(kFull, d);
        const unsigned before = d < 256 ? wcnt[warp][d] : 0u;
        rank[c] = before + __popc(peers & lt);
        __syncwarp();
        if (d < 256 && (peers & lt) == 0u) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();

    // digit tid: offsets of each warp's run within the digit's run, and the tile total
    unsigned int tile_count = 0u;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const unsigned int cnt = wcnt[w][tid];
        wcnt[w][tid] = tile_count;
        tile_count += cnt;
    }
    unsigned long long* my = pub + tile * 256 + tid;
    if (tile == 0) {
        *reinterpret_cast<volatile unsigned long long*>(my) = kFlagInclusive | tile_count;
    } else {
        *reinterpret_cast<volatile unsigned long long*>(my) = kFlagAggregate | tile_count;
    }

    // exclusive scans over the 256 digits (thread tid = digit): the pass's
    // digit counts give the digit's start in the output, the tile's counts
    // the digit's start in the tile's digit order
    const unsigned int hc = hist[tid];
    unsigned int inc = hc, tinc = tile_count;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(kFull, inc, o);
        const unsigned int ty = __shfl_up_sync(kFull, tinc, o);
        if (lane >= o) {
            inc += y;
            tinc += ty;
        }
    }
    __shared__ unsigned int twsum[kWarps];
    if (lane == 31) {
        wsum[warp] = inc;
        twsum[warp] = tinc;
    }
    __syncthreads();
    unsigned long long start = inc - hc;
    unsigned int tst = tinc - tile_count;
    for (int w = 0; w < warp; ++w) {
        start += wsum[w];
        tst += twsum[w];
    }
    tstart[tid] = tst;

    // look back over the tiles before this one
    unsigned long long prefix = 0ull;
    if (tile > 0) {
        long long t = tile - 1;
        unsigned long long t0 = 0ull;
        bool timed = false;
        while (t >= 0) {
            const unsigned long long v = *reinterpret_cast<volatile unsigned long long*>(pub + t * 256 + tid);
            if ((v >> 62) == 0ull) {  // not published yet
                if (!timed) {
                    t0 = globaltimer_ns();
                    timed = true;
                } else if (globaltimer_ns() - t0 > kLookbackLimitNs) {
                    atomicExch(status, kStatusTimeout);
                    break;
                }
                continue;
            }
            timed = false;
            prefix += v & kCountMask;
            if ((v >> 62) == 2ull) break;
            --t;
        }
        *reinterpret_cast<volatile unsigned long long*>(my) = kFlagInclusive | (prefix + tile_count);
    }
    gshift[tid] = (long long)(start + prefix) - (long long)tst;
    __syncthreads();

    // the tile in digit order in shared memory, then out in that order
#pragma unroll
    for (int c = 0; c < kItems; ++c) {
        const int d = digit(c);
        if (d < 256) {
            const unsigned int at = tstart[d] + wcnt[warp][d] + rank[c];
            skey[at] = key[c];
            sval[at] = val[c];
        }
    }
    __syncthreads();
    const long long rem = count - tile * kTile;
    const int tile_n = rem < kTile ? (int)rem : kTile;
    for (int e = tid; e < tile_n; e += kThreads) {
        const unsigned long long k2 = skey[e];
        const int d = (int)((k2 >> shift) & 0xFFull);
        const long long pos = gshift[d] + e;
        kout[pos] = k2;
        vout[pos] = sval[e];
    }
}

int passes_for(int bits) { return (bits + 7) / 8; }

long long tiles_for(long long count) { return (count + kTile - 1) / kTile; }

}  // namespace

size_t radix_sort_temp_bytes(long long count, int bits) {
    const int P = passes_for(bits > 0 ? bits : 1);
    const long long tiles = tiles_for(count > 0 ? count : 1);
    // published words (8-byte aligned first), digit counts, tile counters
    return (size_t)P * (size_t)tiles * 256 * sizeof(unsigned long long) + (size_t)P * 256 * sizeof(unsigned int) +
           (size_t)P * sizeof(unsigned int);
}

cudaError_t radix_sort_pairs(unsigned long long* keys, float* vals, unsigned long long* keys_tmp, float* vals_tmp,
                             long long count, int bits, void* temp, size_t temp_bytes, int32_t* status,
                             cudaStream_t s, unsigned long long** keys_out, float** vals_out, int* launches,
                             const unsigned long long* count_dev) {
    *keys_out = keys;
    *vals_out = vals;
    if (count <= 1 || bits <= 0) return cudaSuccess;
    if (bits > 8 * kMaxPasses) return cudaErrorInvalidValue;
    const int P = passes_for(bits);
    const long long tiles = tiles_for(count);
    const size_t need = radix_sort_temp_bytes(count, bits);
    if (temp_bytes < need) return cudaErrorInvalidValue;
    unsigned long long* pub = static_cast<unsigned long long*>(temp);
    unsigned int* hist = reinterpret_cast<unsigned int*>(pub + (size_t)P * tiles * 256);
    unsigned int* tile_ctr = hist + P * 256;
    cudaError_t e = cudaMemsetAsync(temp, 0, need, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes)) !=
        cudaSuccess)
        return e;
    long long hgrid = (count + kThreads * 16 - 1) / (kThreads * 16);
    if (hgrid > device_sm_count() * 8) hgrid = device_sm_count() * 8;
    hist_all_kernel<<<(unsigned)hgrid, kThreads, 0, s>>>(keys, count, P, hist, count_dev);
    if (launches) *launches += 1;
    unsigned long long *ka = keys, *kb = keys_tmp;
    float *va = vals, *vb = vals_tmp;
    for (int p = 0; p < P; ++p) {
        onesweep_kernel<<<(unsigned)tiles, kThreads, kStageBytes, s>>>(ka, va, kb, vb, count, 8 * p, hist + p * 256,
                                                                       tile_ctr + p, pub + (size_t)p * tiles * 256,
                                                                       status, count_dev);
        if (launches) *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
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
