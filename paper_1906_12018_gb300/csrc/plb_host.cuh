// Host-side helpers of the build drivers (undirected: plb_build.cu;
// directed: plb_directed.cu; weighted: plb_weighted.cu): device allocations
// of one build, CUDA-event timers, launch geometry, the last CUDA error of
// this thread.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <initializer_list>
#include <vector>

#include "plb_round.cuh"

namespace plb {

constexpr int kFlatThreads = 256;
constexpr int kGpWarpThreads = 256;

// Device allocations of one build (stream-ordered, from the library pool),
// all returned when the build ends.
struct DevPool {
    cudaStream_t s;
    std::vector<void*> ptrs;
    bool failed = false;
    explicit DevPool(cudaStream_t st) : s(st) {}
    template <typename T>
    T* alloc(int64_t count) {
        void* p = nullptr;
        const size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
        if (plb::dev_alloc(&p, bytes, s) != cudaSuccess) {
            (void)cudaGetLastError();
            failed = true;
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    void release(void* p) {
        auto it = std::find(ptrs.begin(), ptrs.end(), p);
        if (it != ptrs.end()) {
            cudaFreeAsync(p, s);
            ptrs.erase(it);
        }
    }
    // Frees every allocation except those in keep (stream-ordered).
    void release_all_except(std::initializer_list<const void*> keep) {
        std::vector<void*> kept;
        for (void* p : ptrs) {
            if (std::find(keep.begin(), keep.end(), p) != keep.end()) kept.push_back(p);
            else cudaFreeAsync(p, s);
        }
        ptrs.swap(kept);
    }
    ~DevPool() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
};

// CUDA-event spans per kernel class (profile option).
struct Timer {
    bool on;
    cudaStream_t s;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[8];
    std::vector<cudaEvent_t> all;  // every event once (spans may share an end point)
    explicit Timer(bool enabled, cudaStream_t st) : on(enabled), s(st) {}
    cudaEvent_t mark() {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        all.push_back(e);
        return e;
    }
    void span(int cls, cudaEvent_t a, cudaEvent_t b) { ev[cls].push_back({a, b}); }
    double total(int cls) {
        double t = 0;
        for (auto& p : ev[cls]) {
            float ms = 0;
            cudaEventElapsedTime(&ms, p.first, p.second);
            t += ms;
        }
        return t;
    }
    ~Timer() {
        for (cudaEvent_t e : all) cudaEventDestroy(e);
        (void)cudaGetLastError();
    }
};
enum { T_PREP = 0, T_FRONT = 1, T_GPW = 2, T_GPB = 3, T_GPG = 4, T_MERGE = 5, T_FINAL = 6, T_ALL = 7 };

inline int grid_for(int64_t items, int threads, int max_blocks) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

inline int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 132;
    }
    return sms;
}

inline int pow2_at_least(int64_t x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Dynamic shared memory of k_gp_block in bytes, in the order the kernel
// carves it up: scalars (48 words) + warp sums (34) + histogram (256) +
// top-hub masks + prefix per thread + 64-bit row start per thread + set (also
// kByteStage per warp of byte-map staging) + map + candidate list (limit +
// 32 per warp) + byte map.
inline size_t gp_block_smem_bytes(int bthr, int log_s, int log_m, int cand_limit) {
    return sizeof(uint32_t) * (48 + 34 + 256 + kTopRow + (size_t)((bthr + 2) & ~1) + 2 * (size_t)bthr +
                               ((size_t)1 << log_s) + ((size_t)1 << log_m) + (size_t)cand_limit + (size_t)bthr +
                               kByteHubs / 4);
}

// Records the failing CUDA call for plb_last_error (this thread).
void set_last_error(cudaError_t e, int line);

}  // namespace plb
