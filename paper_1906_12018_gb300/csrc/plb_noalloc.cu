// Allocation-free variant of plb_degree_order.
//
// Some callers cannot let a library allocate device memory: processes whose
// device memory is owned by a host framework's allocator (so every byte is
// accounted for there), serving loops that admit work by a fixed HBM budget,
// and latency-critical paths where cudaMalloc/cudaFree may block or
// synchronise the device.  This entry point sorts in a fixed scratch array
// that lives in the library image instead of allocating one per call.
#include <mutex>

#include "plb_internal.cuh"

namespace plb {

cudaError_t degree_order_with_scratch(const int64_t* row_ptr, int64_t n, int32_t* order, uint64_t* keys,
                                      int64_t n2, cudaStream_t s);

namespace {

// Sort keys of up to PLB_NOALLOC_MAX_VERTICES vertices (8 bytes each, 8 MiB).
// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) uint64_t g_noalloc_keys[PLB_NOALLOC_MAX_VERTICES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint64_t* g_keys_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code may not use the array's name as a device pointer).
cudaError_t scratch_for_current_device(uint64_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_keys_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_keys);
        if (e != cudaSuccess) return e;
        g_keys_ptr[dev] = static_cast<uint64_t*>(p);
    }
    *out = g_keys_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace plb

extern "C" int plb_degree_order_noalloc(const plb_csr* g, int32_t* order_out, plb_stream stream) {
    if (!g || g->n < 0 || (g->n > 0 && (!g->row_ptr || !order_out))) return PLB_ERR_INVALID;
    if (g->n > PLB_NOALLOC_MAX_VERTICES) return PLB_ERR_TOO_LARGE;
    if (g->n == 0) return PLB_OK;
    (void)cudaGetLastError();
    uint64_t* keys = nullptr;
    if (plb::scratch_for_current_device(&keys) != cudaSuccess) {
        (void)cudaGetLastError();
        return PLB_ERR_CUDA;
    }
    int64_t n2 = 1;
    while (n2 < g->n) n2 <<= 1;
    // every key slot [0, n2) is rewritten by the call before it is read
    const cudaError_t e = plb::degree_order_with_scratch(g->row_ptr, g->n, order_out, keys, n2,
                                                         (cudaStream_t)stream);
    return e == cudaSuccess ? PLB_OK : PLB_ERR_CUDA;
}
