// gumap_knn_run_noalloc: the kNN lists of every vertex through the MS-BFS
// kernel, with all of its scratch taken from one fixed array that lives in
// this file, so the call itself allocates nothing.
//
// Why it exists: some callers cannot call cudaMalloc at the point where they
// need kNN lists -- code running under a framework that owns all device
// memory (a caching allocator or a fixed memory budget), or a latency-bound
// loop where cudaMalloc/cudaFree and their implicit device synchronisation
// are not acceptable. They pass the graph and the output buffers; the
// library contributes only this array.
//
// The array is a file-scope __device__ variable of kNoallocScratchBytes
// (16 MiB): every GPU that loads the library holds it until the process
// exits. In host code its name is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress once per device (the first
// call on that device, with the device current) and then passed to the
// kernels. That first call should come before any stream capture.
//
// All calls share the array and it keeps the previous call's contents:
// every part that must start at zero is cleared on the call's stream before
// use. Two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and give undefined results.
#include "gumap.h"
#include "gumap_internal.cuh"

#include <algorithm>
#include <mutex>

namespace gumap {

namespace {

constexpr size_t kNoallocScratchBytes = 16ull << 20;
constexpr int kMaxDevices = 64;
constexpr size_t kAlign = 256;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct DeviceSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
    int coop_grid = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Bytes the scratch needs for n vertices and S sources per block.
size_t scratch_bytes(int32_t n, int S) {
    const size_t W = (size_t)S / 32;
    return align_up(sizeof(DeviceCounters)) + align_up(W * 4) + align_up(W * 4) + align_up((size_t)S * 4) +
           align_up((size_t)n * 4) + 3 * (size_t)n * W * 4;
}

}  // namespace

}  // namespace gumap

using namespace gumap;

extern "C" int gumap_knn_run_noalloc(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                                     int32_t k, int mode, int32_t* out_idx, uint16_t* out_dist,
                                     int32_t* status_out, void* stream) {
    report_error(GUMAP_OK, "");
    if (!row_ptr || (!col_idx && nnz > 0) || !out_idx || !out_dist)
        return report_error(GUMAP_ERR_INVALID_ARG, "NULL CSR or output pointer");
    if (n < 2 || nnz < 0 || nnz > 0x7FFFFFFFll) return report_error(GUMAP_ERR_INVALID_ARG, "n or nnz out of range");
    if (k < 1 || k > GUMAP_MAX_K || k > n - 1) return report_error(GUMAP_ERR_INVALID_ARG, "k must be in [1, min(n-1, 256)]");
    if (mode != GUMAP_FULL && mode != GUMAP_PARTIAL) return report_error(GUMAP_ERR_INVALID_ARG, "bad mode");
    if (scratch_bytes(n, 128) > kNoallocScratchBytes)
        return report_error(GUMAP_ERR_TOO_LARGE, "the graph's scratch exceeds the fixed 16 MiB array");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report_error(GUMAP_ERR_CUDA, "no current CUDA device");
    DeviceSetup setup;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        DeviceSetup& s = g_setup[dev];
        if (!s.ready) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
                return report_error(GUMAP_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return report_error(GUMAP_ERR_CUDA, "device attribute query failed");
            const int per_sm = msbfs_max_blocks_per_sm(256);
            if (per_sm <= 0) return report_error(GUMAP_ERR_CUDA, "the MS-BFS kernel cannot be resident");
            s.scratch = static_cast<unsigned char*>(p);
            s.coop_grid = sms * per_sm;
            s.ready = true;
        }
        setup = s;
    }

    // widest source block (multiple of 128, at most the rounded-up n) that fits
    int S = (int)std::min<long long>(((long long)n + 127) / 128 * 128, 1 << 16);
    while (S > 128 && scratch_bytes(n, S) > kNoallocScratchBytes) S -= 128;
    const int W = S / 32;

    unsigned char* p = setup.scratch;
    DeviceCounters* ctr = reinterpret_cast<DeviceCounters*>(p);
    p += align_up(sizeof(DeviceCounters));
    uint32_t* act = reinterpret_cast<uint32_t*>(p);
    p += align_up((size_t)W * 4);
    uint32_t* need = reinterpret_cast<uint32_t*>(p);
    p += align_up((size_t)W * 4);
    int32_t* cnt = reinterpret_cast<int32_t*>(p);
    p += align_up((size_t)S * 4);
    int32_t* order = reinterpret_cast<int32_t*>(p);
    p += align_up((size_t)n * 4);
    uint32_t* bits = reinterpret_cast<uint32_t*>(p);
    const size_t words = (size_t)n * W;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ctr, 0, sizeof(DeviceCounters), st) != cudaSuccess)
        return report_error(GUMAP_ERR_CUDA, "clearing the counters failed");
    if (launch_identity(order, n, st) != cudaSuccess)  // sources and pull order
        return report_error(GUMAP_ERR_CUDA, "identity launch failed");
    const int nblocks = (n + S - 1) / S;
    for (int b = 0; b < nblocks; ++b) {
        MsbfsArgs a{};
        a.row_ptr = row_ptr;
        a.col = col_idx;
        a.n = n;
        a.src = order + (size_t)b * S;
        a.identity = 1;  // order holds 0 .. n-1
        a.src_lo = b * S;
        a.nb = std::min<int32_t>(S, n - b * S);
        a.W = W;
        a.F = bits;
        a.N = bits + words;
        a.S = bits + 2 * words;
        a.heavy = order;
        a.n_heavy = 0;
        a.light = order;
        a.n_light = n;
        a.act = act;
        a.need = need;
        a.cnt = cnt;
        a.out_idx = out_idx + (size_t)b * S * k;
        a.out_dist = out_dist + (size_t)b * S * k;
        a.k = k;
        a.partial = mode == GUMAP_PARTIAL ? 1 : 0;
        a.ctr = ctr;
        a.direction = 1;  // pull only: the push levels' queues would need more scratch
        if (cudaMemsetAsync(ctr, 0, kLaunchCounterBytes, st) != cudaSuccess)
            return report_error(GUMAP_ERR_CUDA, "clearing the launch counters failed");
        // as many CTAs as the block's items need, at most the resident grid
        if (launch_msbfs(a, msbfs_grid_for(a, setup.coop_grid), 256, st) != cudaSuccess)
            return report_error(GUMAP_ERR_CUDA, "msbfs launch failed");
    }
    if (status_out &&
        cudaMemcpyAsync(status_out, &ctr->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return report_error(GUMAP_ERR_CUDA, "copying the status word failed");
    return GUMAP_OK;
}
