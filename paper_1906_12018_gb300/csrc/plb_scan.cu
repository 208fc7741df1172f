// Device-wide exclusive prefix sum of int64 values (the append/compaction
// step of each round turns per-vertex counts into row offsets with it).
//
// Three phases per level: each 256-thread block scans a tile of 2048 values
// in shared memory and records the tile total; the tile totals are scanned
// (recursively); the tile offsets are added back.
#include "plb_internal.cuh"

namespace plb {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr int kTile = kThreads * kPerThread;

// Block-wide exclusive scan of each thread's partial sum.
__device__ int64_t block_excl_scan(int64_t x, int64_t* sh_warp, int64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < kThreads / 32 ? sh_warp[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kThreads / 32) sh_warp[lane] = wi - w;
        if (lane == kThreads / 32 - 1) sh_warp[kThreads / 32] = wi;
    }
    __syncthreads();
    const int64_t r = sh_warp[wid] + incl - x;
    *total = sh_warp[kThreads / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads) k_scan_tiles(const int64_t* in, int64_t* out, int64_t n,
                                                         int64_t* tile_sums, const int* skip) {
    __shared__ int64_t sh_warp[kThreads / 32 + 1];
    if (skip && *skip) return;
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPerThread;
    int64_t v[kPerThread];
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        sum += v[k];
    }
    int64_t total;
    int64_t run = block_excl_scan(sum, sh_warp, &total);
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads) k_scan_add(int64_t* out, int64_t n, const int64_t* tile_offs,
                                                       const int* skip) {
    if (skip && *skip) return;
    const int64_t add = tile_offs[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int k = threadIdx.x; k < kTile; k += kThreads) {
        const int64_t i = base + k;
        if (i < n) out[i] += add;
    }
}

// single-tile scan writing out[n] = total
__global__ void __launch_bounds__(kThreads) k_scan_single(const int64_t* in, int64_t* out, int64_t n,
                                                          const int* skip) {
    __shared__ int64_t sh_warp[kThreads / 32 + 1];
    if (skip && *skip) return;
    const int64_t base = (int64_t)threadIdx.x * kPerThread;
    int64_t v[kPerThread];
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        sum += v[k];
    }
    int64_t total;
    int64_t run = block_excl_scan(sum, sh_warp, &total);
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) out[n] = total;
}

__global__ void k_scan_total(int64_t* dst, const int64_t* src, const int* skip) {
    if (skip && *skip) return;
    *dst = *src;
}

}  // namespace

int64_t scan_scratch_elems(int64_t n) {
    int64_t total = 0;
    while (n > kTile) {
        const int64_t t = (n + kTile - 1) / kTile;
        total += t + 1;
        n = t;
    }
    return total + 1;
}

// Kernel launches of one exclusive_scan_i64 over n values.
int scan_launch_count(int64_t n) {
    if (n <= kTile) return 1;
    return 3 + scan_launch_count((n + kTile - 1) / kTile);
}

// out[0..n] = exclusive scan of in[0..n), out[n] = sum.  With skip, every
// kernel returns at once while *skip is non-zero (graph-driven rounds after
// the loop has finished).
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* scratch, cudaStream_t s,
                               const int* skip) {
    if (n <= kTile) {
        k_scan_single<<<1, kThreads, 0, s>>>(in, out, n, skip);
        return cudaGetLastError();
    }
    const int64_t tiles = (n + kTile - 1) / kTile;
    int64_t* sums = scratch;  // tiles + 1 entries
    k_scan_tiles<<<(unsigned)tiles, kThreads, 0, s>>>(in, out, n, sums, skip);
    cudaError_t e = exclusive_scan_i64(sums, sums, tiles, scratch + tiles + 1, s, skip);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)tiles, kThreads, 0, s>>>(out, n, sums, skip);
    k_scan_total<<<1, 1, 0, s>>>(out + n, sums + tiles, skip);  // total = sums[tiles]
    return cudaGetLastError();
}

}  // namespace plb
