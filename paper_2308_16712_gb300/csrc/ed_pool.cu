// ed_pool.cu -- a library-private, stream-ordered device memory pool for the
// arrays the library allocates itself: the solvers' work vectors, the basis
// build's temporaries and the large arrays of a basis.  cudaMalloc / cudaFree
// of gigabytes take milliseconds and synchronise the device; memory freed back
// to this pool is kept (up to a release threshold, min(8 GiB, 1/16 of the
// device memory), applied at synchronisation points) and handed out again by
// the next call without either cost.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "ed_kernels.cuh"

namespace edk {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaError_t device_pool(cudaMemPool_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if ((e = cudaMemPoolCreate(&p, &props)) != cudaSuccess)
            return e;
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        uint64_t keep = std::min<uint64_t>(8ull << 30, total_b / 16);
        if ((e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pools[dev] = p;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

}  // namespace

cudaError_t ws_alloc(void **p, size_t bytes, cudaStream_t s)
{
    cudaMemPool_t pool;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess)
        return e;
    return cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 1), pool, s);
}

cudaError_t ws_free(void *p, cudaStream_t s)
{
    return p ? cudaFreeAsync(p, s) : cudaSuccess;
}

size_t ws_cached_bytes()
{
    cudaMemPool_t pool;
    if (device_pool(&pool) != cudaSuccess)
        return 0;
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess)
        return 0;
    return reserved > used ? (size_t)(reserved - used) : 0;
}

}  // namespace edk

extern "C" ed_status ed_release_cached_memory(void)
{
    std::lock_guard<std::mutex> lock(edk::g_pool_mutex);
    for (cudaMemPool_t p : edk::g_pools)
        if (p && cudaMemPoolTrimTo(p, 0) != cudaSuccess)
            return ED_ERR_CUDA;
    return ED_OK;
}
