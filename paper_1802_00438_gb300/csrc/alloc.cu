// Every device and pinned-host allocation the library makes goes through dev_malloc /
// host_malloc, so that
//   - a test can make the n-th next allocation fail as if the device were out of memory
//     (allocation-failure injection from the host: no GPU fault, nothing launched), and check
//     that the call that made it reports ST_ERR_OOM and releases what it had allocated;
//   - stencil_debug_live_allocs() counts what the library holds, so a test sees a leak as a
//     count that does not return to its starting value.
#include <cuda_runtime.h>

#include <atomic>

#include "../../include/stencil.h"
#include "internal.h"

namespace stn {
namespace {

std::atomic<int> g_fail_in{0};          // > 0: the allocation that brings it to 0 fails
std::atomic<long long> g_live{0};       // allocations made and not yet freed

// true when this allocation is the armed one (the counter then disarms itself)
bool injected_failure()
{
    int n = g_fail_in.load(std::memory_order_relaxed);
    while (n > 0) {
        if (g_fail_in.compare_exchange_weak(n, n - 1, std::memory_order_relaxed))
            return n == 1;
    }
    return false;
}

}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live.fetch_add(1, std::memory_order_relaxed);
    return e;
}

void dev_free(void *p)
{
    if (p && cudaFree(p) == cudaSuccess) g_live.fetch_sub(1, std::memory_order_relaxed);
}

cudaError_t host_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) g_live.fetch_add(1, std::memory_order_relaxed);
    return e;
}

void host_free(void *p)
{
    if (p && cudaFreeHost(p) == cudaSuccess) g_live.fetch_sub(1, std::memory_order_relaxed);
}

}  // namespace stn

extern "C" {

int stencil_debug_fail_alloc(int n)
{
    if (n < 0) return ST_ERR_INVALID_ARG;
    stn::g_fail_in.store(n, std::memory_order_relaxed);
    return ST_OK;
}

long long stencil_debug_live_allocs(void) { return stn::g_live.load(std::memory_order_relaxed); }

}  // extern "C"
