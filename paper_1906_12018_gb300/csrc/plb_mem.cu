// Device memory of the library: one stream-ordered pool per device that keeps
// freed blocks for reuse (repeated builds and queries do not return memory to
// the driver and map it again).  plb_release_cached_memory trims the pools.
#include <mutex>

#include "plb_internal.cuh"

namespace plb {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaError_t pool_for_current_device(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool;
    cudaError_t e = pool_for_current_device(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

}  // namespace plb

extern "C" int plb_release_cached_memory(void) {
    if (cudaDeviceSynchronize() != cudaSuccess) {
        (void)cudaGetLastError();
        return PLB_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(plb::g_pool_mu);
    for (int d = 0; d < plb::kMaxDevices; ++d)
        if (plb::g_pools[d] && cudaMemPoolTrimTo(plb::g_pools[d], 0) != cudaSuccess) {
            (void)cudaGetLastError();
            return PLB_ERR_CUDA;
        }
    return PLB_OK;
}

extern "C" int plb_memory_stats(int64_t* out, int reset) {
    if (!out) return PLB_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= plb::kMaxDevices) {
        (void)cudaGetLastError();
        return PLB_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(plb::g_pool_mu);
    cudaMemPool_t pool = plb::g_pools[dev];
    for (int i = 0; i < 4; ++i) out[i] = 0;
    if (!pool) return PLB_OK;
    const cudaMemPoolAttr attrs[4] = {cudaMemPoolAttrUsedMemCurrent, cudaMemPoolAttrUsedMemHigh,
                                      cudaMemPoolAttrReservedMemCurrent, cudaMemPoolAttrReservedMemHigh};
    for (int i = 0; i < 4; ++i) {
        uint64_t v = 0;
        if (cudaMemPoolGetAttribute(pool, attrs[i], &v) != cudaSuccess) {
            (void)cudaGetLastError();
            return PLB_ERR_CUDA;
        }
        out[i] = (int64_t)v;
    }
    if (reset) {  // high marks can only be set to 0, which restarts them from the current use
        uint64_t zero = 0;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess ||
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReservedMemHigh, &zero) != cudaSuccess) {
            (void)cudaGetLastError();
            return PLB_ERR_CUDA;
        }
    }
    return PLB_OK;
}
