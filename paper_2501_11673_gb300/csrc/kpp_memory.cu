// kpp_memory.cu -- the library's device memory: a cache of long-lived buffers and a stream-ordered pool.
//
// Long-lived buffers (block factors, inverses, memos, solver states, the device copies of host inputs)
// come from dev_malloc and go back through dev_free.  A released buffer is not handed back to the
// driver: it waits on a free list keyed by (device, size) for the next request of that size.  A solve
// repeated on one shape (a factor phase per request, a benchmark step) then maps its gigabytes once
// instead of on every call; mapping and unmapping several GiB costs milliseconds of host time during
// which the GPU idles.  dev_free synchronises the device first, as cudaFree does, so that a buffer is
// never handed out again while a kernel may still read it.  The free list holds at most a quarter of
// the device's memory; a release beyond that goes to the driver.
//
// Short-lived scratch comes from dev_malloc_async: a pool per device owned by the library, whose release
// threshold keeps freed memory mapped across synchronisations.  (The device's default pool returns
// freed memory to the driver at every synchronisation, and the next request maps it again.)
//
// kpp_device_cache_trim returns both caches to the driver; kpp_device_cache_bytes reports what they
// hold.  Every request is counted (kpp_device_alloc_count), served from a cache or not.
#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <unordered_map>

#include "../../include/kpp.h"
#include "kpp_runtime.h"

namespace kpp {

namespace {

constexpr int MAX_DEV = 64;

struct Block {
    int dev;
    size_t bytes;
};

std::mutex g_mu;
std::unordered_map<void *, Block> g_live;              // buffers handed out by dev_malloc
std::multimap<std::pair<int, size_t>, void *> g_free;  // (device, size) -> released buffer
size_t g_free_bytes[MAX_DEV] = {};
cudaMemPool_t g_pool[MAX_DEV] = {};
std::atomic<unsigned long long> g_allocs{0};

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

size_t cache_cap(int dev) {
    static size_t cap[MAX_DEV] = {};
    if (!cap[dev]) {
        size_t fr = 0, tot = 0;
        cap[dev] = (cudaMemGetInfo(&fr, &tot) == cudaSuccess && tot) ? tot / 4 : ((size_t)16 << 30);
    }
    return cap[dev];
}

// Return the free list of device `dev` to the driver (g_mu held).
void trim_free_list(int dev) {
    for (auto it = g_free.begin(); it != g_free.end();) {
        if (it->first.first == dev) {
            cudaFree(it->second);
            g_free_bytes[dev] -= it->first.second;
            it = g_free.erase(it);
        } else {
            ++it;
        }
    }
}

cudaMemPool_t pool_for(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps pr = {};
        pr.allocType = cudaMemAllocationTypePinned;
        pr.handleTypes = cudaMemHandleTypeNone;
        pr.location.type = cudaMemLocationTypeDevice;
        pr.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &pr) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = p;
    }
    return g_pool[dev];
}

}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    const int dev = current_device();
    if (dev < 0 || dev >= MAX_DEV) return cudaMalloc(p, bytes);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_free.find({dev, bytes});
        if (it != g_free.end()) {
            *p = it->second;
            g_free.erase(it);
            g_free_bytes[dev] -= bytes;
            g_live[*p] = Block{dev, bytes};
            return cudaSuccess;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        // the free list may hold what the request needs: give it back and try once more
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> lk(g_mu);
            trim_free_list(dev);
        }
        e = cudaMalloc(p, bytes);
    }
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_live[*p] = Block{dev, bytes};
    }
    return e;
}

void dev_free(void *p) {
    if (!p) return;
    Block b{-1, 0};
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_live.find(p);
        if (it != g_live.end()) {
            b = it->second;
            g_live.erase(it);
        }
    }
    if (b.dev < 0) {  // not from dev_malloc
        cudaFree(p);
        return;
    }
    // as cudaFree: no kernel may still use the buffer once it can be handed out again
    int cur = current_device();
    if (cur != b.dev) cudaSetDevice(b.dev);
    const bool idle = cudaDeviceSynchronize() == cudaSuccess;
    bool cached = false;
    if (idle) {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_free_bytes[b.dev] + b.bytes <= cache_cap(b.dev)) {
            g_free.insert({{b.dev, b.bytes}, p});
            g_free_bytes[b.dev] += b.bytes;
            cached = true;
        }
    }
    if (!cached) cudaFree(p);
    if (cur != b.dev) cudaSetDevice(cur);
}

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    const int dev = current_device();
    cudaMemPool_t pool = (dev >= 0 && dev < MAX_DEV) ? pool_for(dev) : nullptr;
    if (!pool) return cudaMallocAsync(p, bytes, st);
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        cudaMemPoolTrimTo(pool, 0);
        {
            std::lock_guard<std::mutex> lk(g_mu);
            trim_free_list(dev);
        }
        e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    }
    return e;
}

unsigned long long dev_alloc_requests() { return g_allocs.load(std::memory_order_relaxed); }

// High-priority streams for work that other kernels should not hold up (the factor phase's Cholesky,
// which the inverses and the memo of finished blocks fill in around): lent out and returned, so that
// concurrent callers each get their own and none is created per call.
namespace {
std::multimap<int, cudaStream_t> g_streams;  // device -> idle stream
}

cudaStream_t priority_stream_acquire() {
    const int dev = current_device();
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_streams.find(dev);
        if (it != g_streams.end()) {
            cudaStream_t h = it->second;
            g_streams.erase(it);
            return h;
        }
    }
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    cudaStream_t h = nullptr;
    if (cudaStreamCreateWithPriority(&h, cudaStreamNonBlocking, hi) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return h;
}

void priority_stream_release(cudaStream_t h) {
    if (!h) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_streams.insert({current_device(), h});
}

}  // namespace kpp

using namespace kpp;

extern "C" {

size_t kpp_device_cache_bytes(void) {
    const int dev = current_device();
    if (dev < 0 || dev >= MAX_DEV) return 0;
    size_t held = 0;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        held = g_free_bytes[dev];
        pool = g_pool[dev];
    }
    if (pool) {
        uint64_t reserved = 0, used = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
            held += (size_t)(reserved - used);
    }
    return held;
}

kpp_status kpp_device_cache_trim(void) {
    clear_error();
    const int dev = current_device();
    if (dev < 0 || dev >= MAX_DEV) return KPP_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        set_error("kpp_device_cache_trim: cudaDeviceSynchronize: %s", cudaGetErrorString(cudaGetLastError()));
        return KPP_ERR_CUDA;
    }
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        trim_free_list(dev);
        pool = g_pool[dev];
    }
    if (pool && cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
        set_error("kpp_device_cache_trim: cudaMemPoolTrimTo failed");
        return KPP_ERR_CUDA;
    }
    return KPP_OK;
}

}  // extern "C"
