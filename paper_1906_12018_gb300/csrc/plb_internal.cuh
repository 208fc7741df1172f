// Internal device/host helpers of the labeling library (sm_103a).
//
// Label entries are packed 32-bit words: bits 31..8 = hub rank (24 bits),
// bits 7..0 = distance.  Within a row, entries are sorted by hub rank, so a
// plain unsigned comparison of packed words orders them by hub (hubs are
// unique per row).  0xFFFFFFFF never occurs as an entry (distance 255 is
// reserved) and marks empty hash slots.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "plb.h"

namespace plb {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kHubShift = 8;

__host__ __device__ __forceinline__ uint32_t pack(uint32_t hub, uint32_t d) { return (hub << kHubShift) | d; }
__host__ __device__ __forceinline__ uint32_t hub_of(uint32_t e) { return e >> kHubShift; }
__host__ __device__ __forceinline__ uint32_t dist_of(uint32_t e) { return e & 0xFFu; }

// frontier row descriptor: start (40 bits) | count (24 bits)
__host__ __device__ __forceinline__ uint64_t fpack(uint64_t start, uint32_t cnt) { return (start << 24) | cnt; }
__host__ __device__ __forceinline__ uint64_t fstart(uint64_t x) { return x >> 24; }
__host__ __device__ __forceinline__ uint32_t fcount(uint64_t x) { return (uint32_t)(x & 0xFFFFFFu); }

// Fibonacci hashing of a hub rank into a table of 2^logcap slots.
__device__ __forceinline__ uint32_t hslot(uint32_t key, int logcap) {
    return (key * 0x9E3779B1u) >> (32 - logcap);
}

// Insert key into an open-addressing set; returns true if it was new.
// The caller guarantees the table never fills (load <= 1/2 plus the number
// of concurrently inserting threads).
// (Every probe loop below is bounded by the table size, so a table broken by
// a bug can never spin a kernel forever.)
__device__ __forceinline__ bool set_insert(uint32_t* tab, int logcap, uint32_t key) {
    const uint32_t mask = (1u << logcap) - 1u;
    uint32_t s = hslot(key, logcap);
    for (uint32_t i = 0; i <= mask; ++i) {
        const uint32_t old = atomicCAS(tab + s, kEmpty, key);
        if (old == kEmpty) return true;
        if (old == key) return false;
        s = (s + 1) & mask;
    }
    return false;
}

// Insert a packed label entry keyed by its hub (keys unique by construction).
__device__ __forceinline__ void map_insert(uint32_t* tab, int logcap, uint32_t e) {
    const uint32_t mask = (1u << logcap) - 1u;
    uint32_t s = hslot(hub_of(e), logcap);
    for (uint32_t i = 0; i <= mask && atomicCAS(tab + s, kEmpty, e) != kEmpty; ++i) s = (s + 1) & mask;
}

// Distance stored for hub w, or 0xFFFFFFFF when w is not in the map.
__device__ __forceinline__ uint32_t map_find(const uint32_t* tab, int logcap, uint32_t w) {
    const uint32_t mask = (1u << logcap) - 1u;
    uint32_t s = hslot(w, logcap);
    for (uint32_t i = 0; i <= mask; ++i) {
        const uint32_t x = tab[s];
        if (x == kEmpty) return kEmpty;
        if (hub_of(x) == w) return dist_of(x);
        s = (s + 1) & mask;
    }
    return kEmpty;
}

__device__ __forceinline__ int warp_incl_scan(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += t;
    }
    return x;
}

// Runs of equal keys over the lanes (each key's lanes consecutive, as the
// rows of consecutive arcs): returns, in every lane, the sum of x over the
// lane's run, which holds lanes *first..*last.  All 32 lanes call it.
__device__ __forceinline__ int run_sum(int64_t key, int x, int lane, int* first, int* last) {
    const int incl = warp_incl_scan(x, lane);
    const int64_t kprev = __shfl_up_sync(kFull, key, 1);
    const int64_t knext = __shfl_down_sync(kFull, key, 1);
    const unsigned starts = __ballot_sync(kFull, lane == 0 || kprev != key);
    const unsigned ends = __ballot_sync(kFull, lane == 31 || knext != key);
    const int f = 31 - __clz(starts & (0xFFFFFFFFu >> (31 - lane)));  // last run start at or below the lane
    const int l = __ffs(ends & (0xFFFFFFFFu << lane)) - 1;            // first run end at or above it
    const int before = __shfl_sync(kFull, incl - x, f);
    *first = f;
    *last = l;
    return __shfl_sync(kFull, incl, l) - before;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// Largest lane k whose exclusive prefix excl_k <= item (excl non-decreasing
// over lanes).  All 32 lanes must call.
__device__ __forceinline__ int warp_owner(int excl, int item) {
    int k = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int e = __shfl_sync(kFull, excl, k + step);
        if (e <= item) k += step;
    }
    return k;
}

// Number of entries of sorted a[0..len) that are < key (hub comparison on
// packed entries when the key is given as a packed word with distance 0).
__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t* a, int64_t len, uint32_t key) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Row r of offsets off[] containing item p (largest r with off[r] <= p) in [lo, hi].
__device__ __forceinline__ int64_t row_of(const int64_t* off, int64_t lo, int64_t hi, int64_t p) {
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Bitonic sort of a[0..P) (P a power of two) by a group of nthreads threads.
// Each step runs over the P/2 compare-exchange pairs (i, i + j), i the pair
// index t with a zero bit inserted at bit log2(j): no idle half of the
// threads.
template <typename Sync>
__device__ void group_bitonic_sort(uint32_t* a, int P, int tid, int nthreads, Sync sync) {
    const int half = P >> 1;
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = tid; t < half; t += nthreads) {
                const int i = 2 * t - (t & (j - 1));
                const int l = i + j;
                const uint32_t x = a[i], y = a[l];
                const bool up = (i & k) == 0;
                if ((x > y) == up) {
                    a[i] = y;
                    a[l] = x;
                }
            }
            sync();
        }
    }
}

__host__ __device__ __forceinline__ int ceil_log2_i64(int64_t x) {
    int b = 0;
    while ((int64_t(1) << b) < x) ++b;
    return b;
}

}  // namespace plb

// ---------------------------------------------------------------- host side
struct plb_labels {
    int64_t n = 0;
    int64_t total = 0;
    int64_t* off = nullptr;        // n+1, by original id
    uint32_t* packed = nullptr;    // total, (hub rank << 8) | dist, rows sorted by hub
    uint32_t* hub = nullptr;       // total
    uint8_t* dist = nullptr;       // total
    int32_t* order = nullptr;      // n, rank -> id
    int32_t max_dist = 0;
    int32_t rounds = 0;
    int64_t bytes = 0;
    plb_build_stats stats{};
    void* shared = nullptr;        // storage shared by the sets of one batched build
};

namespace plb {

// Stream-ordered allocation from the library's per-device pool (freed with
// cudaFreeAsync, or cudaFree after synchronising).
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);

// Device-wide exclusive scan of int64 values; out may alias in.
// count(i) is evaluated for i in [0, n) and out[n] receives the total.
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* block_sums,
                               cudaStream_t s, const int* skip = nullptr);
int64_t scan_scratch_elems(int64_t n);
int scan_launch_count(int64_t n);

}  // namespace plb
