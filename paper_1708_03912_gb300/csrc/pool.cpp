// Caching allocator for the library's device and pinned host buffers.
//
// Handles are cheap to create and destroy in a loop (one mesh per step): their tables,
// workspaces and pinned scalars come from per-device free lists instead of cudaMalloc /
// cudaMallocHost, and go back to the lists when the handle is destroyed (after the device
// has been synchronised, so nothing in flight still uses them).  A request reuses the
// smallest cached block of at least its size and at most twice its size (sizes rounded up
// to 256 bytes); otherwise a new block is allocated.  When an allocation fails for lack of
// memory, the cached blocks of that device are released and the allocation is retried.
// fl_pool_trim releases every cached block; fl_pool_stats reports the cache.
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <unordered_map>

#include "context.h"

namespace fl {
namespace {

constexpr int MAX_DEV = 64;

struct Pool {
    std::mutex mu;
    std::multimap<size_t, void*> free_dev[MAX_DEV];
    std::multimap<size_t, void*> free_host;
    std::unordered_map<void*, std::pair<size_t, int>> live_dev;  // block -> (size, device)
    std::unordered_map<void*, size_t> live_host;
    int64_t cached_dev = 0, cached_host = 0, hits = 0, misses = 0;
};

Pool& pool() {
    static Pool* p = new Pool;  // never destroyed: blocks may be returned during process exit
    return *p;
}

size_t round_size(size_t bytes) { return ((bytes < 256 ? 256 : bytes) + 255) / 256 * 256; }

// take a cached block of [bytes, 2 bytes] from m, or nullptr
void* take(std::multimap<size_t, void*>& m, size_t bytes, size_t* got) {
    auto it = m.lower_bound(bytes);
    if (it == m.end() || it->first > 2 * bytes) return nullptr;
    void* p = it->second;
    *got = it->first;
    m.erase(it);
    return p;
}

void release_dev_locked(Pool& P, int dev) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    for (auto& kv : P.free_dev[dev]) {
        cudaFree(kv.second);
        P.cached_dev -= (int64_t)kv.first;
    }
    P.free_dev[dev].clear();
    if (cur != dev) cudaSetDevice(cur);
}

}  // namespace

cudaError_t pool_dev_alloc(void** out, size_t bytes) {
    *out = nullptr;
    bytes = round_size(bytes);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= MAX_DEV) return cudaMalloc(out, bytes);
    Pool& P = pool();
    std::lock_guard<std::mutex> lk(P.mu);
    size_t got = 0;
    if (void* p = take(P.free_dev[dev], bytes, &got)) {
        P.cached_dev -= (int64_t)got;
        P.hits++;
        P.live_dev[p] = {got, dev};
        *out = p;
        return cudaSuccess;
    }
    P.misses++;
    cudaError_t e = cudaMalloc(out, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        release_dev_locked(P, dev);
        e = cudaMalloc(out, bytes);
    }
    if (e != cudaSuccess) {
        *out = nullptr;
        return e;
    }
    P.live_dev[*out] = {bytes, dev};
    return cudaSuccess;
}

void pool_dev_free(void* p) {
    if (!p) return;
    Pool& P = pool();
    std::lock_guard<std::mutex> lk(P.mu);
    auto it = P.live_dev.find(p);
    if (it == P.live_dev.end()) {
        cudaFree(p);  // not from the pool
        return;
    }
    const size_t bytes = it->second.first;
    const int dev = it->second.second;
    P.live_dev.erase(it);
    P.free_dev[dev].emplace(bytes, p);
    P.cached_dev += (int64_t)bytes;
}

cudaError_t pool_host_alloc(void** out, size_t bytes) {
    *out = nullptr;
    bytes = round_size(bytes);
    Pool& P = pool();
    std::lock_guard<std::mutex> lk(P.mu);
    size_t got = 0;
    if (void* p = take(P.free_host, bytes, &got)) {
        P.cached_host -= (int64_t)got;
        P.hits++;
        P.live_host[p] = got;
        *out = p;
        return cudaSuccess;
    }
    P.misses++;
    cudaError_t e = cudaMallocHost(out, bytes);
    if (e != cudaSuccess) {
        *out = nullptr;
        return e;
    }
    P.live_host[*out] = bytes;
    return cudaSuccess;
}

void pool_host_free(void* p) {
    if (!p) return;
    Pool& P = pool();
    std::lock_guard<std::mutex> lk(P.mu);
    auto it = P.live_host.find(p);
    if (it == P.live_host.end()) {
        cudaFreeHost(p);
        return;
    }
    const size_t bytes = it->second;
    P.live_host.erase(it);
    P.free_host.emplace(bytes, p);
    P.cached_host += (int64_t)bytes;
}

}  // namespace fl

extern "C" {

int64_t fl_pool_trim(void) {
    fl::Pool& P = fl::pool();
    std::lock_guard<std::mutex> lk(P.mu);
    const int64_t released = P.cached_dev + P.cached_host;
    for (int d = 0; d < fl::MAX_DEV; ++d)
        if (!P.free_dev[d].empty()) fl::release_dev_locked(P, d);
    for (auto& kv : P.free_host) cudaFreeHost(kv.second);
    P.free_host.clear();
    P.cached_host = 0;
    return released;
}

void fl_pool_stats(int64_t* cached_device_bytes, int64_t* cached_host_bytes, int64_t* hits, int64_t* misses) {
    fl::Pool& P = fl::pool();
    std::lock_guard<std::mutex> lk(P.mu);
    if (cached_device_bytes) *cached_device_bytes = P.cached_dev;
    if (cached_host_bytes) *cached_host_bytes = P.cached_host;
    if (hits) *hits = P.hits;
    if (misses) *misses = P.misses;
}

}  // extern "C"
