// mem.cu -- every device and page-locked host allocation the library makes,
// with an optional process-wide budget (vc_set_memory_limit).
//
// The budget lets a process that shares its GPU (or its pinned host memory)
// with another framework bound what this library takes, and makes the
// library's out-of-memory paths reachable on purpose: an allocation that would
// exceed the budget fails with cudaErrorMemoryAllocation before any CUDA call,
// exactly as a refused cudaMalloc would, and the caller reports VC_ENOMEM.
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace {

struct Pool {
    std::unordered_map<void *, size_t> sizes;
    u64 used = 0, limit = 0;  // limit 0: unlimited
};

std::mutex g_mu;
Pool g_dev, g_host;

bool reserve(Pool &p, size_t n)
{
    if (p.limit && (n > p.limit || p.used > p.limit - n)) return false;
    p.used += n;
    return true;
}

void record(Pool &p, void *ptr, size_t n)
{
    p.sizes[ptr] = n;
}

void release(Pool &p, void *ptr)
{
    auto it = p.sizes.find(ptr);
    if (it == p.sizes.end()) return;
    p.used -= it->second;
    p.sizes.erase(it);
}

}  // namespace

cudaError_t lib_malloc(void **p, size_t n)
{
    *p = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (!reserve(g_dev, n)) return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, n);
    std::lock_guard<std::mutex> g(g_mu);
    if (e != cudaSuccess) {
        g_dev.used -= n;
        *p = nullptr;
        return e;
    }
    record(g_dev, *p, n);
    return cudaSuccess;
}

cudaError_t lib_free(void *p)
{
    if (!p) return cudaSuccess;
    {
        std::lock_guard<std::mutex> g(g_mu);
        release(g_dev, p);
    }
    return cudaFree(p);
}

cudaError_t lib_host_alloc(void **p, size_t n, unsigned flags)
{
    *p = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (!reserve(g_host, n)) return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaHostAlloc(p, n, flags);
    std::lock_guard<std::mutex> g(g_mu);
    if (e != cudaSuccess) {
        g_host.used -= n;
        *p = nullptr;
        return e;
    }
    record(g_host, *p, n);
    return cudaSuccess;
}

cudaError_t lib_free_host(void *p)
{
    if (!p) return cudaSuccess;
    {
        std::lock_guard<std::mutex> g(g_mu);
        release(g_host, p);
    }
    return cudaFreeHost(p);
}

extern "C" vc_status vc_set_memory_limit(uint64_t device_bytes, uint64_t pinned_bytes)
{
    std::lock_guard<std::mutex> g(g_mu);
    g_dev.limit = device_bytes;
    g_host.limit = pinned_bytes;
    return VC_OK;
}

extern "C" vc_status vc_get_memory_usage(uint64_t *device_bytes, uint64_t *pinned_bytes)
{
    if (!device_bytes && !pinned_bytes) return VC_EINVAL;
    std::lock_guard<std::mutex> g(g_mu);
    if (device_bytes) *device_bytes = g_dev.used;
    if (pinned_bytes) *pinned_bytes = g_host.used;
    return VC_OK;
}
