// Device-memory pool of the library's handles.
//
// gumap_knn_destroy returns its buffers here instead of calling cudaFree
// (which synchronises the whole device), and gumap_knn_create / run take
// buffers of the same rounded size back, so a caller that creates and
// destroys handles per request pays for allocation once. Blocks are cached
// per device and rounded size (powers of two below 1 MiB, whole MiB above)
// up to a cap (GUMAP_POOL_BYTES, default 8 GiB); beyond the cap a freed
// block goes back to CUDA. The caller of pool_free guarantees the device no
// longer uses the block (the handle synchronised its device first).
#include "gumap.h"
#include "gumap_internal.cuh"

#include <cstdlib>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

namespace gumap {

namespace {

std::mutex g_pool_mutex;
std::multimap<std::pair<int, size_t>, void*> g_free;  // (device, rounded size) -> block
size_t g_cached = 0;
size_t g_cap = 0;
bool g_cap_set = false;

size_t round_size(size_t b) {
    if (b == 0) b = 1;
    if (b >= (1u << 20)) return (b + (1u << 20) - 1) / (1u << 20) * (1u << 20);
    size_t p = 256;
    while (p < b) p <<= 1;
    return p;
}

size_t cap_bytes() {
    if (!g_cap_set) {
        g_cap_set = true;
        g_cap = 8ull << 30;
        if (const char* e = std::getenv("GUMAP_POOL_BYTES")) g_cap = (size_t)std::strtoull(e, nullptr, 10);
    }
    return g_cap;
}

}  // namespace

int device_sm_count() {
    static std::mutex mu;
    static std::vector<int> cache;  // per device ordinal; 0 = not queried yet
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    std::lock_guard<std::mutex> lk(mu);
    if ((size_t)dev >= cache.size()) cache.resize((size_t)dev + 1, 0);
    if (cache[(size_t)dev] <= 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 1;
        cache[(size_t)dev] = sms;
    }
    return cache[(size_t)dev];
}

cudaError_t pool_alloc(void** p, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t r = round_size(bytes);
    {
        std::lock_guard<std::mutex> lk(g_pool_mutex);
        auto it = g_free.find({dev, r});
        if (it != g_free.end()) {
            *p = it->second;
            g_free.erase(it);
            g_cached -= r;
            return cudaSuccess;
        }
    }
    e = cudaMalloc(p, r);
    if (e == cudaErrorMemoryAllocation) {  // give the cache back to CUDA and retry once
        pool_trim(dev);
        cudaGetLastError();
        e = cudaMalloc(p, r);
    }
    return e;
}

void pool_free(void* p, size_t bytes) {
    if (!p) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    const size_t r = round_size(bytes);
    {
        std::lock_guard<std::mutex> lk(g_pool_mutex);
        if (g_cached + r <= cap_bytes()) {
            g_free.emplace(std::make_pair(dev, r), p);
            g_cached += r;
            return;
        }
    }
    cudaFree(p);
}

void pool_trim(int device) {
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto it = g_free.begin(); it != g_free.end();) {
        if (device < 0 || it->first.first == device) {
            cudaSetDevice(it->first.first);
            cudaFree(it->second);
            g_cached -= it->first.second;
            it = g_free.erase(it);
        } else {
            ++it;
        }
    }
    cudaSetDevice(cur);
}

size_t pool_cached_bytes() {
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    return g_cached;
}

}  // namespace gumap

extern "C" int gumap_pool_trim(int device) {
    gumap::pool_trim(device);
    return GUMAP_OK;
}

extern "C" int64_t gumap_pool_cached_bytes(void) { return (int64_t)gumap::pool_cached_bytes(); }
