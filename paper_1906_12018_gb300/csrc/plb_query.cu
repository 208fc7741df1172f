// Batched 2-hop distance queries (Sec. 2.1):
//   Dis(s, t) = min over hubs h in L(s) and L(t) of d(s,h) + d(h,t).
// One warp per pair: lanes stride over the shorter of the two hub-sorted rows
// and binary-search each hub in the longer row; a warp min-reduction gives
// the answer.
#include <algorithm>

#include "plb_internal.cuh"

namespace plb {
namespace {

constexpr int kQThreads = 256;
constexpr int kMaxSets = 128;

struct SetDesc {
    const int64_t* off;
    const uint32_t* packed;
    int64_t n;
};

struct SetTable {
    SetDesc s[kMaxSets];
};

// Rows: s in the set (off_s, ent_s), t in (off_t, ent_t); the same set for
// undirected labels, L_out and L_in for directed ones (d(s -> t)).
__device__ __forceinline__ int32_t answer_pair2(const int64_t* off_s, const uint32_t* ent_s, const int64_t* off_t,
                                                const uint32_t* ent_t, int64_t n, int32_t s, int32_t t, int lane) {
    if (s < 0 || t < 0 || (int64_t)s >= n || (int64_t)t >= n) return PLB_BAD_PAIR;
    const uint32_t* ent = ent_s;
    const uint32_t* ent2 = ent_t;
    int64_t ab = off_s[s], al = off_s[s + 1] - ab;
    int64_t bb = off_t[t], bl = off_t[t + 1] - bb;
    if (al > bl) {
        const uint32_t* e = ent;
        ent = ent2;
        ent2 = e;
        int64_t x = ab;
        ab = bb;
        bb = x;
        x = al;
        al = bl;
        bl = x;
    }
    uint32_t best = 0xFFFFFFFFu;
    for (int64_t j = lane; j < al; j += 32) {
        const uint32_t x = ent[ab + j];
        const uint32_t key = pack(hub_of(x), 0);
        const int64_t pos = lower_bound_u32(ent2 + bb, bl, key);
        if (pos < bl) {
            const uint32_t y = ent2[bb + pos];
            if (hub_of(y) == hub_of(x)) best = min(best, dist_of(x) + dist_of(y));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFull, best, o));
    return best == 0xFFFFFFFFu ? PLB_UNREACHABLE : (int32_t)best;
}

__device__ __forceinline__ int32_t answer_pair(const int64_t* off, const uint32_t* ent, int64_t n, int32_t s,
                                               int32_t t, int lane) {
    return answer_pair2(off, ent, off, ent, n, s, t, lane);
}

__global__ void __launch_bounds__(kQThreads) k_query2(const int64_t* off_s, const uint32_t* ent_s,
                                                      const int64_t* off_t, const uint32_t* ent_t, int64_t n,
                                                      const int32_t* pairs, int64_t q, int32_t* out) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < q; i += nw) {
        const int32_t r = answer_pair2(off_s, ent_s, off_t, ent_t, n, pairs[2 * i], pairs[2 * i + 1], lane);
        if (lane == 0) out[i] = r;
    }
}

__global__ void __launch_bounds__(kQThreads) k_query(const int64_t* off, const uint32_t* ent, int64_t n,
                                                     const int32_t* pairs, int64_t q, int32_t* out) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < q; i += nw) {
        const int32_t s = pairs[2 * i], t = pairs[2 * i + 1];
        const int32_t r = answer_pair(off, ent, n, s, t, lane);
        if (lane == 0) out[i] = r;
    }
}

__global__ void __launch_bounds__(kQThreads) k_query_multi(SetTable tab, int set_lo, int set_hi, int64_t m,
                                                           const int32_t* set_idx, const int32_t* pairs, int64_t q,
                                                           int32_t* out) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < q; i += nw) {
        const int32_t k = set_idx[i];
        if (k < 0 || (int64_t)k >= m) {
            if (set_lo == 0 && lane == 0) out[i] = PLB_BAD_PAIR;
            continue;
        }
        if (k < set_lo || k >= set_hi) continue;
        const SetDesc& d = tab.s[k - set_lo];
        const int32_t r = answer_pair(d.off, d.packed, d.n, pairs[2 * i], pairs[2 * i + 1], lane);
        if (lane == 0) out[i] = r;
    }
}

int query_grid(int64_t q) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 132;
    }
    int64_t blocks = (q * 32 + kQThreads - 1) / kQThreads;
    const int64_t cap = (int64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

}  // namespace
}  // namespace plb

extern "C" int plb_query_batch(const plb_labels* L, const int32_t* pairs, int64_t q, int32_t* dist_out,
                               plb_stream stream) {
    if (!L || q < 0 || (q > 0 && (!pairs || !dist_out))) return PLB_ERR_INVALID;
    if (q == 0) return PLB_OK;
    (void)cudaGetLastError();
    plb::k_query<<<plb::query_grid(q), plb::kQThreads, 0, (cudaStream_t)stream>>>(L->off, L->packed, L->n, pairs, q,
                                                                                  dist_out);
    return cudaGetLastError() == cudaSuccess ? PLB_OK : PLB_ERR_CUDA;
}

extern "C" int plb_query_directed(const plb_labels* L_out, const plb_labels* L_in, const int32_t* pairs, int64_t q,
                                  int32_t* dist_out, plb_stream stream) {
    if (!L_out || !L_in || L_out->n != L_in->n || q < 0 || (q > 0 && (!pairs || !dist_out))) return PLB_ERR_INVALID;
    if (q == 0) return PLB_OK;
    (void)cudaGetLastError();
    plb::k_query2<<<plb::query_grid(q), plb::kQThreads, 0, (cudaStream_t)stream>>>(
        L_out->off, L_out->packed, L_in->off, L_in->packed, L_out->n, pairs, q, dist_out);
    return cudaGetLastError() == cudaSuccess ? PLB_OK : PLB_ERR_CUDA;
}

extern "C" int plb_query_multi(const plb_labels* const* sets, int64_t m, const int32_t* set_idx, const int32_t* pairs,
                               int64_t q, int32_t* dist_out, plb_stream stream) {
    if (m < 0 || q < 0 || (m > 0 && !sets) || (q > 0 && (!pairs || !dist_out || !set_idx))) return PLB_ERR_INVALID;
    for (int64_t k = 0; k < m; ++k)
        if (!sets[k]) return PLB_ERR_INVALID;
    if (q == 0) return PLB_OK;
    (void)cudaGetLastError();
    const int grid = plb::query_grid(q);
    for (int64_t lo = 0; lo < std::max<int64_t>(m, 1); lo += plb::kMaxSets) {
        plb::SetTable tab{};
        const int64_t hi = std::min<int64_t>(m, lo + plb::kMaxSets);
        for (int64_t k = lo; k < hi; ++k) tab.s[k - lo] = {sets[k]->off, sets[k]->packed, sets[k]->n};
        plb::k_query_multi<<<grid, plb::kQThreads, 0, (cudaStream_t)stream>>>(tab, (int)lo, (int)hi, m, set_idx, pairs,
                                                                              q, dist_out);
        if (cudaGetLastError() != cudaSuccess) return PLB_ERR_CUDA;
    }
    return PLB_OK;
}
