// Degree order (Sec. 6.1: vertices ordered by degree, the heuristic of the
// original PLL): rank -> id with degree descending and ties by smaller id.
// Keys (0x7FFFFFFF - degree) << 32 | id are unique, so any correct sort
// gives the same order; a bitonic network over a power-of-two padded key
// array sorts them (tiles of 2048 keys in shared memory, longer strides in
// global memory).
#include "plb_internal.cuh"

namespace plb {
namespace {

constexpr int kSortTile = 2048;
constexpr int kSortThreads = 1024;

__global__ void k_deg_keys(const int64_t* row_ptr, int64_t n, int64_t n2, uint64_t* keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = ~0ull;
        if (i < n) {
            const int64_t deg = row_ptr[i + 1] - row_ptr[i];
            k = ((uint64_t)(0x7FFFFFFFll - deg) << 32) | (uint64_t)i;
        }
        keys[i] = k;
    }
}

__device__ __forceinline__ void cswap(uint64_t* a, int i, int l, bool up) {
    const uint64_t x = a[i], y = a[l];
    if ((x > y) == up) {
        a[i] = y;
        a[l] = x;
    }
}

// Full bitonic sort of each tile (stages k = 2 .. tile), directions taken
// from the global index so that the tiles feed the global merge stages.
__global__ void __launch_bounds__(kSortThreads) k_sort_tiles(uint64_t* keys, int tile) {
    __shared__ uint64_t sk[kSortTile];
    const int64_t base = (int64_t)blockIdx.x * tile;
    for (int i = threadIdx.x; i < tile; i += blockDim.x) sk[i] = keys[base + i];
    __syncthreads();
    for (int k = 2; k <= tile; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < tile; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) cswap(sk, i, l, ((base + i) & k) == 0);
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < tile; i += blockDim.x) keys[base + i] = sk[i];
}

// One global compare-exchange step (stride j >= tile) of merge stage k.
__global__ void k_sort_global_step(uint64_t* keys, int64_t n2, int64_t j, int64_t k) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = i ^ j;
        if (l > i) {
            const uint64_t x = keys[i], y = keys[l];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
                keys[i] = y;
                keys[l] = x;
            }
        }
    }
}

// Remaining strides j < tile of merge stage k, inside each tile.
__global__ void __launch_bounds__(kSortThreads) k_sort_tile_merge(uint64_t* keys, int tile, int64_t k) {
    __shared__ uint64_t sk[kSortTile];
    const int64_t base = (int64_t)blockIdx.x * tile;
    for (int i = threadIdx.x; i < tile; i += blockDim.x) sk[i] = keys[base + i];
    __syncthreads();
    for (int j = tile >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < tile; i += blockDim.x) {
            const int l = i ^ j;
            if (l > i) cswap(sk, i, l, ((base + i) & k) == 0);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < tile; i += blockDim.x) keys[base + i] = sk[i];
}

__global__ void k_keys_to_order(const uint64_t* keys, int64_t n, int32_t* order) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        order[r] = (int32_t)(keys[r] & 0xFFFFFFFFull);
}

}  // namespace

// Sorts keys[0..n2) ascending (n2 a power of two).
cudaError_t bitonic_sort_u64(uint64_t* keys, int64_t n2, cudaStream_t s) {
    const int tile = (int)(n2 < kSortTile ? n2 : kSortTile);
    const int64_t tiles = n2 / tile;
    k_sort_tiles<<<(unsigned)tiles, kSortThreads, 0, s>>>(keys, tile);
    for (int64_t k = 2 * (int64_t)tile; k <= n2; k <<= 1) {
        for (int64_t j = k >> 1; j >= tile; j >>= 1) {
            int64_t blocks = (n2 + 255) / 256;
            if (blocks > 65535) blocks = 65535;
            k_sort_global_step<<<(unsigned)blocks, 256, 0, s>>>(keys, n2, j, k);
        }
        k_sort_tile_merge<<<(unsigned)tiles, kSortThreads, 0, s>>>(keys, tile, k);
    }
    return cudaGetLastError();
}

cudaError_t degree_order_with_scratch(const int64_t* row_ptr, int64_t n, int32_t* order, uint64_t* keys,
                                      int64_t n2, cudaStream_t s) {
    int64_t blocks = (n2 + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_deg_keys<<<(unsigned)blocks, 256, 0, s>>>(row_ptr, n, n2, keys);
    cudaError_t e = bitonic_sort_u64(keys, n2, s);
    if (e != cudaSuccess) return e;
    k_keys_to_order<<<(unsigned)blocks, 256, 0, s>>>(keys, n, order);
    return cudaGetLastError();
}

}  // namespace plb

extern "C" int plb_degree_order(const plb_csr* g, int32_t* order_out, plb_stream stream) {
    if (!g || g->n < 0 || (g->n > 0 && (!g->row_ptr || !order_out))) return PLB_ERR_INVALID;
    if (g->n >= PLB_MAX_VERTICES) return PLB_ERR_TOO_LARGE;
    if (g->n == 0) return PLB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t n2 = 1;
    while (n2 < g->n) n2 <<= 1;
    uint64_t* keys = nullptr;
    if (plb::dev_alloc((void**)&keys, sizeof(uint64_t) * n2, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return PLB_ERR_OOM;
    }
    const cudaError_t e = plb::degree_order_with_scratch(g->row_ptr, g->n, order_out, keys, n2, s);
    cudaFreeAsync(keys, s);
    return e == cudaSuccess ? PLB_OK : PLB_ERR_CUDA;
}
