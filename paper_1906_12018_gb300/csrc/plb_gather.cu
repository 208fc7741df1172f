// Gather + prune kernels of rounds d >= 2 (Alg. 3, Sec. 3.1): for every
// receiver v, the unique messages of round d (hubs h < v of the neighbours'
// frontier rows dL_{d-1}, not already hubs of v) and the distance check of
// each candidate against the labels of round d - 1 (the snapshot: accept
// (h, d) iff no common hub w has d(w, v) + d(w, h) <= d).
//   k_gp_warp   one vertex per warp, tables in shared memory;
//   k_gp_block  one vertex per 256-thread block, any size.
// Both append the accepted hubs to the new frontier: the warp tier sorted,
// the block tier unsorted (it lists those vertices for the row sort).
#include "plb_kernels.cuh"
#include "plb_round.cuh"

namespace plb {
namespace {
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
}  // namespace

// Side B of the check (see check_chunk), per tier (measured: side B saves most
// on power-law graphs with heavy hubs in both tiers).
constexpr int kWarpSideBMin = 16, kWarpSideBShift = 1;
constexpr int kBlockSideBMin = 16, kBlockSideBShift = 1;

// Top-hub witness prefilter for the 32 candidates of a chunk (one per lane):
// candidate h has a witness among the kTopHubs highest-ranked hubs when
// E_i(v) & C_j(h) != 0 for some i >= 1, j = min(d - i, kTopLevels) >= 1, where
// E_i(v) (v's hubs at distance exactly i) is staged in shared memory (ev,
// kTopLevels x kTopWords words) and C_j(h) is h's cumulative mask.  Returns
// the mask of lanes whose candidate is pruned.
__device__ __forceinline__ unsigned top_prefilter(const uint32_t* top, const uint32_t* ev, uint32_t d, uint32_t h,
                                                  bool valid) {
    uint32_t hit = 0;
    if (valid) {
        const uint32_t* th = top + (int64_t)h * kTopRow;
        const int imax = min((int)d - 1, kTopLevels);
        for (int i = 1; i <= imax; ++i) {
            const int j = min((int)d - i, kTopLevels);
            const uint4* cj = reinterpret_cast<const uint4*>(th + (j - 1) * kTopWords);
            const uint32_t* e = ev + (i - 1) * kTopWords;
#pragma unroll
            for (int q = 0; q < kTopWords / 4; ++q) {
                const uint4 a = cj[q];
                hit |= (a.x & e[4 * q]) | (a.y & e[4 * q + 1]) | (a.z & e[4 * q + 2]) | (a.w & e[4 * q + 3]);
            }
        }
    }
    return __ballot_sync(kFull, hit != 0);
}

// Stage E_i(v) = C_i(v) & ~C_{i-1}(v), i = 1..kTopLevels, into ev (cooperative:
// thread t of nthr handles words t, t + nthr, ...).
__device__ __forceinline__ void stage_exact_levels(const uint32_t* top, int32_t v, uint32_t* ev, int t, int nthr) {
    const uint32_t* tv = top + (int64_t)v * kTopRow;
    for (int q = t; q < kTopRow; q += nthr) {
        const uint32_t c = tv[q];
        const uint32_t prev = q >= kTopWords ? tv[q - kTopWords] : 0u;
        ev[q] = c & ~prev;
    }
}

// Distance check of up to 32 candidates held one per lane (valid lanes).
// A witness for candidate h is a hub w of both v and h with
// d(w,v) + d(w,h) <= d (the test of Alg. 3 with the labels of round d-1).
// Each candidate scans one side:
//   A: the entries of L(h) (its last entry, (h,0), is never a witness and is
//      skipped), each looked up in the hub-keyed table M of L(v) (shared
//      memory, or v's row of the global probe index when mv_global);
//   B: the entries of L(v) with hub < h (only those can be hubs of h), each
//      probed in h's row of the global probe index (rows of >= 16 entries).
// B is considered only for |L(h)| >= b_min (the count of L(v)'s hubs below h
// is a binary search in L(v)'s row) and taken when it is the shorter scan, by
// a factor 2^b_shift against a shared-memory M (whose probes are cheaper
// than the global table's).  All (candidate, entry) pairs are spread over
// the lanes; a candidate's remaining entries are skipped once it has a
// witness.  Every candidate first goes through the top-hub prefilter, which
// is exact for the kTopHubs highest-ranked hubs while d <= kTopLevels + 1
// (a witness w has 1 <= d(w,v), d(w,h) <= d - 1): for a candidate it does not
// prune, no top hub is a witness, so both scans start past the top hubs
// (L(h)'s count of them comes with h's check record, L(v)'s is tv_top).
// Returns the lanes whose candidate survives.
__device__ __forceinline__ unsigned check_chunk(const GpParams& p, uint32_t d, const uint32_t* M, int log_m,
                                                bool mv_global, int b_min, int b_shift, const uint32_t* lv,
                                                int64_t lvlen, int tv_top, uint32_t h, bool valid,
                                                unsigned long long& probed, const uint32_t* tv,
                                                unsigned long long& prefiltered, unsigned long long* chk) {
    const int lane = threadIdx.x & 31;
    int64_t base = 0;  // A: first entry of L(h) scanned; B: start of h's probe table
    int items = 0, meta = 0;  // meta: 0 = side A, else log2(table size) + 1
    int skip_b = 0;           // side B: the scan of L(v) starts at this entry
    // h's check record (row bounds and probe-table descriptor: one 16-byte
    // load, one memory sector) is requested before the top-hub prefilter
    // reads h's masks, so the two loads overlap
    uint4 rec = make_uint4(0u, 0u, 0u, 0u);
    if (valid && p.hrec_h) rec = p.hrec_h[h];
    // every candidate first tries the exact top-hub prefilter (one mask row
    // per distance level; a hit settles the candidate without a scan)
    const unsigned pf = top_prefilter(p.top_h, tv, d, h, valid);
    if (lane == 0) prefiltered += __popc(pf);
    const bool pruned = (pf >> lane) & 1u;
    // past the top hubs when the prefilter settles them (see above)
    const bool skip_top = d <= (uint32_t)kTopLevels + 1u;
    if (valid) {
        int64_t hb, he;
        uint64_t hd;
        int top_h = 0;  // entries of L(h) with hub < kTopHubs
        if (p.hrec_h) {
            const uint64_t row = ((uint64_t)rec.y << 32) | rec.x;
            hb = (int64_t)(row >> 24);
            he = hb + (int64_t)(row & 0xFFFFFFu);
            hd = (((uint64_t)rec.w << 32) | rec.z) & kHrecDescMask;
            top_h = (int)(rec.w >> kHrecTopShift);
        } else if (!pruned || p.count_check) {
            hb = p.loff_h[h];
            he = p.loff_h[h + 1];
            hd = p.hdesc_h[h];
        } else {
            hb = he = 0;
            hd = 0;
        }
        const int la = (int)(he - hb) - 1;
        if (p.count_check) {  // the cost model's reads: L(v)'s entries below h, and L(h)
            chk[0] += (unsigned long long)lower_bound_u32(lv, lvlen, pack(h, 0));
            chk[1] += (unsigned long long)(la + 1);
        }
        if (!pruned) {
            const int sa = skip_top ? min(top_h, la) : 0;  // side A starts past L(h)'s top hubs
            base = hb + sa;
            items = la - sa;
            if (la >= b_min && hd) {
                const int lb = (int)lower_bound_u32(lv, lvlen, pack(h, 0));
                const int sb = skip_top ? min(tv_top, lb) : 0;  // side B starts past L(v)'s top hubs
                if (mv_global ? lb - sb < la - sa : ((lb - sb) << b_shift) < la - sa) {
                    items = lb - sb;
                    base = (int64_t)(hd >> 8);
                    meta = (int)(hd & 0xFFu) + 1;  // log2 + 1
                    skip_b = sb;
                }
            }
        }
    }
    if (pruned) valid = false;
    const unsigned vmask = __ballot_sync(kFull, valid);
    const int incl = warp_incl_scan(items, lane);
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - items;
    unsigned pm = 0;  // candidates with a witness so far (the same in every lane)
    // kCheckUnroll items per lane per step: their entry loads (side A: L(h);
    // side B: L(v)) are all issued before any lookup uses one
    for (int ib = 0; ib < total; ib += 32 * kCheckUnroll) {
        if ((pm & vmask) == vmask) break;
        int ku[kCheckUnroll], mku[kCheckUnroll];
        int64_t bku[kCheckUnroll];
        uint32_t xu[kCheckUnroll];
#pragma unroll
        for (int u = 0; u < kCheckUnroll; ++u) {
            const int it = ib + 32 * u + lane;
            const int k = warp_owner(excl, it);
            bku[u] = __shfl_sync(kFull, base, k);
            const int exk = __shfl_sync(kFull, excl, k);
            mku[u] = __shfl_sync(kFull, meta, k);
            const int sbk = __shfl_sync(kFull, skip_b, k);
            ku[u] = (it < total && !((pm >> k) & 1u)) ? k : -1;
            xu[u] = kEmpty;
            if (ku[u] >= 0) xu[u] = mku[u] == 0 ? p.lent_h[bku[u] + (it - exk)] : lv[sbk + (it - exk)];
        }
        unsigned hits = 0;
#pragma unroll
        for (int u = 0; u < kCheckUnroll; ++u) {
            if (ku[u] < 0) continue;
            const uint32_t x = xu[u];
            // side A: x is an entry of L(h), looked up in L(v)'s map; side B:
            // x is an entry of L(v), looked up in h's probe table
            const uint32_t dw = mku[u] == 0 ? map_find(M, log_m, hub_of(x))
                                            : map_find(p.htab_h + bku[u], mku[u] - 1, hub_of(x));
            if (dw != kEmpty && dw + dist_of(x) <= d) hits |= 1u << ku[u];
            ++probed;
        }
        pm |= __reduce_or_sync(kFull, hits);
    }
    return vmask & ~pm;
}

// Gather of v's messages with hub in [lo, hi) (hi <= v: only hubs that
// outrank v) into the set S: the frontier rows dL_{d-1}(a) of the neighbours
// are sorted, so each row's sub-range is found by binary search.  Warp-level
// load-balanced expansion over 32 neighbours at a time.  With M, hubs already
// in L(v) are skipped.  Stops (returns false) when the set would exceed
// `limit` entries.
__device__ __forceinline__ bool gather_range(const GpParams& p, int64_t nb, int64_t ne, int64_t stride, uint32_t lo,
                                             uint32_t hi, uint32_t* S, int log_s, const uint32_t* M, int log_m,
                                             int limit, int* cnt_sm, volatile int* ovf_sm, unsigned long long& msgs) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = nb; base < ne; base += stride) {
        const int64_t j = base + lane;
        int c = 0;
        int64_t st = 0;
        if (j < ne) {
            const int32_t a = p.rcol[j];
            const uint64_t f = p.fse[a];
            const uint32_t n0 = fcount(f);
            if (n0) {
                // the hubs of a frontier row of sender a are <= a (a itself
                // only in round 0): for a < hi the whole row lies below hi
                const uint32_t* row = p.fhub + fstart(f);
                const int64_t a0 = lo ? lower_bound_u32(row, n0, lo) : 0;
                const int64_t a1 = sender_of(p, a) < hi ? (int64_t)n0 : lower_bound_u32(row, n0, hi);
                st = (int64_t)fstart(f) + a0;
                c = (int)(a1 - a0);
            }
        }
        const int incl = warp_incl_scan(c, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - c;
        msgs += (lane == 0) ? (unsigned long long)total : 0ull;
        for (int ib = 0; ib < total; ib += 32 * kGatherUnroll) {
            uint32_t hv[kGatherUnroll];
            // a step inside one row (long rows): every lane reads that row,
            // no per-lane owner search
            const int k1 = warp_owner(excl, ib);
            const int end1 = k1 < 31 ? __shfl_sync(kFull, excl, k1 + 1) : total;
            if (ib + 32 * kGatherUnroll <= end1) {
                const int64_t at = __shfl_sync(kFull, st, k1) + (ib - __shfl_sync(kFull, excl, k1)) + lane;
#pragma unroll
                for (int u = 0; u < kGatherUnroll; ++u) hv[u] = p.fhub[at + 32 * u];
            } else {
#pragma unroll
                for (int u = 0; u < kGatherUnroll; ++u) {
                    const int it = ib + 32 * u + lane;
                    const int k = warp_owner(excl, it);
                    const int64_t stk = __shfl_sync(kFull, st, k);
                    const int exk = __shfl_sync(kFull, excl, k);
                    hv[u] = it < total ? p.fhub[stk + (it - exk)] : kEmpty;
                }
            }
            int nins = 0;
#pragma unroll
            for (int u = 0; u < kGatherUnroll; ++u) {
                const uint32_t h = hv[u];
                if (h != kEmpty && (!M || map_find(M, log_m, h) == kEmpty)) {
                    if (*(volatile int*)cnt_sm >= limit) *ovf_sm = 1;
                    else nins += set_insert(S, log_s, h) ? 1 : 0;
                }
            }
            nins = warp_sum(nins);
            if (lane == 0 && nins) atomicAdd(cnt_sm, nins);
            if (__any_sync(kFull, *ovf_sm != 0)) return false;
        }
    }
    return true;
}

// Block-wide exclusive scan of one int per thread (blockDim <= 1024);
// wsum is shared scratch of 32 ints.  Returns the thread's exclusive prefix
// and the block total in *total.
__device__ __forceinline__ int block_excl_scan(int x, int* wsum, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const int incl = warp_incl_scan(x, lane);
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = lane < nw ? wsum[lane] : 0;
        const int wi = warp_incl_scan(w, lane);
        wsum[lane] = wi - w;
        if (lane == 31) wsum[32] = wi;
    }
    __syncthreads();
    const int r = wsum[wid] + incl - x;
    *total = wsum[32];
    return r;
}

// Shrink the hub range of a pass whose set overflowed: histogram the keys of
// S below hi over 256 buckets of [lo, hi) and cut hi at the first bucket where
// the running count would pass half the capacity.  The kept count is read off
// the histogram; when it fits (always, unless the first bucket alone is too
// full, then the range is narrowed to that bucket and the histogram redone,
// keys at or above hi being ignored), S is rebuilt from the kept keys (C is
// scratch).  All threads call; returns with *hi_sm and *cnt_sm set.
__device__ void shrink_pass(uint32_t* S, int log_s, uint32_t* C, int limit, uint32_t lo, uint32_t* hi_sm,
                            int* cnt_sm, int* hist, int* tmp) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int S_CAP = 1 << log_s;
    while (true) {
        const uint32_t hi = *(volatile uint32_t*)hi_sm;
        const uint32_t bw = (hi - lo + 255u) / 256u;
        for (int b = tid; b < 256; b += nthr) hist[b] = 0;
        __syncthreads();
        for (int sl = tid; sl < S_CAP; sl += nthr) {
            const uint32_t key = S[sl];
            if (key != kEmpty && key < hi) atomicAdd(&hist[(key - lo) / bw], 1);
        }
        __syncthreads();
        if (tid == 0) {
            int cum = 0, b = 0;
            while (b < 255 && cum + hist[b] <= limit / 2) cum += hist[b++];
            if (b == 0) {  // the first bucket alone passes half the capacity: keep it whole
                b = 1;
                cum = hist[0];
            }
            uint32_t nh = lo + (uint32_t)b * bw;
            if (nh > hi) nh = hi;
            *hi_sm = nh;
            tmp[0] = cum;  // keys below nh
            tmp[1] = 0;
        }
        __syncthreads();
        const uint32_t nh = *(volatile uint32_t*)hi_sm;
        const int kept = *(volatile int*)&tmp[0];
        if (kept > limit) continue;  // narrow further (S untouched; keys >= nh are ignored)
        for (int sl = tid; sl < S_CAP; sl += nthr) {
            const uint32_t key = S[sl];
            if (key != kEmpty && key < nh) C[atomicAdd(&tmp[1], 1)] = key;
        }
        __syncthreads();
        for (int sl = tid; sl < S_CAP; sl += nthr) S[sl] = kEmpty;
        __syncthreads();
        for (int q = tid; q < kept; q += nthr) set_insert(S, log_s, C[q]);
        if (tid == 0) *cnt_sm = kept;
        __syncthreads();
        return;
    }
}

// Block-wide load-balanced gather of v's messages with hub in [lo, *hi_sm):
// hubs below W are marked in the byte map B (plain stores: duplicates write
// the same byte, and L(v)'s hubs are cleared afterwards), the others go into
// the set S.  Neighbours are taken in tiles of blockDim; each thread finds its
// neighbour's sub-range of dL_{d-1}(a) (binary searches in the sorted row), a
// block-wide exclusive scan of the counts assigns every thread an equal,
// contiguous share of the tile's messages.  When the set would exceed
// `limit`, its range (hubs >= W) is shrunk (shrink_pass: S keeps the keys
// below the new bound) and every warp resumes its share of the tile from the
// step where it stopped, now dropping hubs at or above the new bound (a later
// pass takes them): no message of the tile is read twice, except those of
// the step that met the overflow.
__device__ void gather_block(const GpParams& p, int64_t nb, int64_t ne, uint32_t lo, uint32_t* hi_sm, uint8_t* B,
                             uint32_t W, uint32_t* S, int log_s, const uint32_t* M, int log_m, int limit, int* cnt_sm,
                             volatile int* ovf_sm, int* wsum, int* sex, int64_t* sst, uint32_t* C, int* hist, int* tmp,
                             unsigned long long& msgs) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nw = nthr >> 5, lane = tid & 31;
    for (int64_t t0 = nb; t0 < ne; t0 += nthr) {
        const uint32_t hi = *(volatile uint32_t*)hi_sm;
        const int64_t j = t0 + tid;
        int c = 0;
        int64_t st = 0;
        if (j < ne) {
            const int32_t a = p.rcol[j];
            const uint64_t f = p.fse[a];
            const uint32_t n0 = fcount(f);
            if (n0) {
                // the hubs of a frontier row of sender a are <= a (a itself
                // only in round 0): for a < hi the whole row lies below hi
                const uint32_t* row = p.fhub + fstart(f);
                const int64_t a0 = lo ? lower_bound_u32(row, n0, lo) : 0;
                const int64_t a1 = sender_of(p, a) < hi ? (int64_t)n0 : lower_bound_u32(row, n0, hi);
                st = (int64_t)fstart(f) + a0;
                c = (int)(a1 - a0);
            }
        }
        // message offsets of the tile's non-empty rows, compacted (rows cut
        // to nothing by the hub range are common and would otherwise be
        // stepped over item by item)
        int total, nne;
        const int excl = block_excl_scan(c, wsum, &total);
        __syncthreads();
        const int fidx = block_excl_scan(c > 0 ? 1 : 0, wsum, &nne);
        if (c > 0) {
            sex[fidx] = excl;
            sst[fidx] = st;
        }
        if (tid == 0) sex[nne] = total;
        __syncthreads();
        // each warp takes a contiguous range of the tile's messages and walks
        // it in windows of 32 rows: lane j holds the start of row k0 + j, and
        // 32 consecutive messages at a time find their row by a warp-shuffle
        // search, so that the lanes of a load read consecutive hubs of a row
        const int per_w = (((total + nw - 1) / nw) + 31) & ~31;
        const int wbeg = (tid >> 5) * per_w, wend = min(total, wbeg + per_w);
        int pos = wbeg;  // this warp's messages before pos are done
        while (true) {
            // hubs at or above hcut are left to a later pass (hcut = hi
            // until the set's range shrinks within this tile)
            const uint32_t hcut = *(volatile uint32_t*)hi_sm;
            if (pos < wend) {
                int k0 = 0, hk = nne - 1;  // row of pos: largest k with sex[k] <= pos
                while (k0 < hk) {
                    const int mid = (k0 + hk + 1) >> 1;
                    if (sex[mid] <= pos) k0 = mid; else hk = mid - 1;
                }
                bool stop = false;
                for (int it0 = pos; it0 < wend && !stop; k0 += 32) {
                    const int kr = k0 + lane;
                    const int ex = kr < nne ? sex[kr] : total;
                    const int64_t stv = kr < nne ? sst[kr] : 0;
                    const int wcap = k0 + 32 < nne ? sex[k0 + 32] : total;
                    const int wend_w = min(wend, wcap);
                    for (int ib = it0; ib < wend_w; ib += 32 * kGatherUnroll) {
                        uint32_t hv[kGatherUnroll];
                        // a step inside one row (long rows): every lane reads
                        // that row, no per-lane owner search
                        const int k1 = warp_owner(ex, ib);
                        const int end1 = k1 < 31 ? __shfl_sync(kFull, ex, k1 + 1) : wcap;
                        if (ib + 32 * kGatherUnroll <= min(end1, wend_w)) {
                            const int64_t at = __shfl_sync(kFull, stv, k1) + (ib - __shfl_sync(kFull, ex, k1)) + lane;
#pragma unroll
                            for (int u = 0; u < kGatherUnroll; ++u) hv[u] = p.fhub[at + 32 * u];
                        } else {
#pragma unroll
                            for (int u = 0; u < kGatherUnroll; ++u) {
                                const int it = ib + 32 * u + lane;
                                const int kk = warp_owner(ex, it);
                                const int exk = __shfl_sync(kFull, ex, kk);
                                const int64_t stk = __shfl_sync(kFull, stv, kk);
                                hv[u] = it < wend_w ? p.fhub[stk + (it - exk)] : kEmpty;
                            }
                        }
                        int nins = 0;
#pragma unroll
                        for (int u = 0; u < kGatherUnroll; ++u) {
                            const uint32_t h = hv[u];
                            if (h < W) {
                                B[h] = 1;
                            } else if (h < hcut && (!M || map_find(M, log_m, h) == kEmpty)) {
                                if (*(volatile int*)cnt_sm >= limit) *ovf_sm = 1;
                                else nins += set_insert(S, log_s, h) ? 1 : 0;
                            }
                        }
                        nins = warp_sum(nins);
                        if (lane == 0 && nins) atomicAdd(cnt_sm, nins);
                        if (__any_sync(kFull, *ovf_sm != 0)) {
                            stop = true;  // resume from this step after the shrink
                            pos = ib;
                            break;
                        }
                    }
                    if (!stop) it0 = wend_w;
                }
                if (!stop) pos = wend;
            }
            __syncthreads();
            // concurrent inserts can pass the limit without raising the flag
            if (*ovf_sm || *(volatile int*)cnt_sm > limit) {
                shrink_pass(S, log_s, C, limit, lo > W ? lo : W, hi_sm, cnt_sm, hist, tmp);  // S holds hubs >= W
                if (tid == 0) *ovf_sm = 0;
                __syncthreads();
                continue;  // every warp resumes at its pos with the smaller range
            }
            break;
        }
        if (tid == 0) msgs += total;
        __syncthreads();  // sex / sst are rewritten by the next tile
    }
}

// One warp per vertex (tables in shared memory):
//  1. stage L(v) into the hub-keyed map M (or, with few candidates against a
//     long row, look L(v) up in v's row of the global probe index);
//  2. gather the unique messages into the set S;
//  3. compact S in place (L(v)'s sorted row behind it when it fits) and
//     check the candidates 32 at a time;
//  4. sort the accepted hubs and append them to the new frontier.
// A vertex whose unique candidates exceed cand_limit goes to the block tier.
__global__ void __launch_bounds__(256, 3) k_gp_warp(GpParams p) {
    extern __shared__ uint32_t sm[];
    const int lane = lane_id(), wib = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int S_CAP = 1 << p.log_s, M_CAP = 1 << p.log_m;
    int* wsc = reinterpret_cast<int*>(sm) + wib * 4;  // [0] unique count [1] overflow
    uint32_t* tvs = sm + 4 * nwarps;                   // per warp: v's exact-distance top-hub masks
    uint32_t* S = tvs + nwarps * kTopRow + wib * (S_CAP + M_CAP);
    uint32_t* M = S + S_CAP;
    unsigned long long c_arcs = 0, c_msgs = 0, c_uniq = 0, c_staged = 0, c_probed = 0, c_acc = 0, c_vert = 0;
    unsigned long long c_pref = 0, c_chk[2] = {0, 0};
    if (p.ctr->done) return;
    const uint32_t d = p.ctr->d;
    const int nlist = *p.list_n;
    for (int i = blockIdx.x * nwarps + wib; i < nlist; i += gridDim.x * nwarps) {
        __syncwarp();
        const int32_t v = p.list[i];
        const int64_t lb = p.loff[v], ll = p.loff[v + 1] - lb;
        // tables sized for this vertex: the set for its candidate bound (when
        // within the tier's limit), the map for |L(v)| (load <= 1/2)
        const uint32_t bnd = p.rbound[v];
        const int log_s = bnd <= (uint32_t)p.cand_limit ? max(5, ceil_log2_i64(2 * (int64_t)bnd)) : p.log_s;
        // L(v) lookups: the map staged in shared memory, or, for a receiver
        // with few candidates against a long (indexed) row, v's row of the
        // global probe index, which saves staging the whole row
        const uint64_t hdv = (p.stage_ratio > 0 && ll >= kIndexMinLen &&
                              (int64_t)bnd * p.stage_ratio < ll) ? p.hdesc[v] : 0ull;
        const bool mglob = hdv != 0;
        const int log_m = mglob ? (int)(hdv & 0xFFu) : max(5, ceil_log2_i64(2 * ll));
        const uint32_t* Mv = mglob ? p.htab + (hdv >> 8) : M;
        for (int s = lane; s < (1 << log_s); s += 32) S[s] = kEmpty;
        if (!mglob)
            for (int s = lane; s < (1 << log_m); s += 32) M[s] = kEmpty;
        if (lane == 0) {
            wsc[0] = 0;
            wsc[1] = 0;
        }
        __syncwarp();
        if (!mglob)
            for (int64_t j = lane; j < ll; j += 32) map_insert(M, log_m, p.lent[lb + j]);
        __syncwarp();
        const int64_t nb = p.roff[v], ne = p.roff[v + 1];
        const bool ok = gather_range(p, nb, ne, 32, 0u, (uint32_t)v, S, log_s, Mv, log_m, p.cand_limit, &wsc[0],
                                     (volatile int*)&wsc[1], c_msgs);
        __syncwarp();
        const int nS = *(volatile int*)&wsc[0];
        if (!ok || nS > p.cand_limit) {
            if (lane == 0) {
                const int o = atomicAdd(p.esc_n, 1);
                p.esc[o] = v;
            }
            continue;
        }
        if (lane == 0) {
            c_arcs += ne - nb;
            c_staged += mglob ? 0 : ll;
            c_vert += 1;
            c_uniq += nS;
        }
        // compact the set in place (write position never passes the read position)
        int nc = 0;
        for (int sb = 0; sb < (1 << log_s); sb += 32) {
            const uint32_t h = S[sb + lane];
            __syncwarp();
            const bool has = h != kEmpty;
            const unsigned m = __ballot_sync(kFull, has);
            if (has) S[nc + __popc(m & ((1u << lane) - 1u))] = h;
            nc += __popc(m);
        }
        __syncwarp();
        // L(v)'s sorted row, copied behind the candidates (the set's slots
        // past nc are free now) when it fits: the checks' binary searches in
        // L(v) and their side-B scans of it then read shared memory
        const uint32_t* lvp = p.lent + lb;
        if (nc > 0 && (int64_t)nc + ll <= S_CAP) {
            uint32_t* lvs = S + (S_CAP - ll);
            for (int64_t j = lane; j < ll; j += 32) lvs[j] = p.lent[lb + j];
            lvp = lvs;
        }
        // entries of L(v) with hub below kTopHubs (the checks' side B starts past them)
        const int lv_top = nc > 0 ? (int)lower_bound_u32(lvp, ll, pack((uint32_t)kTopHubs, 0)) : 0;
        // distance checks, 32 candidates at a time; survivors compacted in place
        uint32_t* tv = tvs + wib * kTopRow;
        if (nc > 0) stage_exact_levels(p.top, v, tv, lane, 32);
        __syncwarp();
        int nacc = 0;
        for (int cb = 0; cb < nc; cb += 32) {
            const bool valid = cb + lane < nc;
            const uint32_t h = valid ? S[cb + lane] : 0u;
            __syncwarp();
            const unsigned okm = check_chunk(p, d, Mv, log_m, mglob, kWarpSideBMin, kWarpSideBShift, lvp, ll, lv_top,
                                             h, valid, c_probed, tv, c_pref, c_chk);
            if ((okm >> lane) & 1u) S[nacc + __popc(okm & ((1u << lane) - 1u))] = h;
            nacc += __popc(okm);
            __syncwarp();
        }
        // the new row leaves sorted by hub rank: bitonic sort of S[0, nacc)
        // (nacc <= cand_limit, a power of two at most half the set's slots)
        if (nacc > 1) {
            if (nacc <= 32) {
                uint32_t x = lane < nacc ? S[lane] : kEmpty;
#pragma unroll
                for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        const uint32_t y = __shfl_xor_sync(kFull, x, j);
                        const bool up = (lane & k) == 0, lower = (lane & j) == 0;
                        x = (lower == up) ? min(x, y) : max(x, y);
                    }
                }
                if (lane < nacc) S[lane] = x;
            } else {
                int P = 64;
                while (P < nacc) P <<= 1;
                for (int j = nacc + lane; j < P; j += 32) S[j] = kEmpty;
                __syncwarp();
                group_bitonic_sort(S, P, lane, 32, WarpSync());
            }
            __syncwarp();
        }
        if (nacc > 0) {
            unsigned long long start = 0;
            if (lane == 0)
                start = p.ostart ? (unsigned long long)p.ostart[v]
                                 : atomicAdd(&p.ctr->cursor, (unsigned long long)nacc);
            start = __shfl_sync(kFull, start, 0);
            if (start + nacc <= p.fcap) {
                for (int j = lane; j < nacc; j += 32) p.fhub_new[start + j] = S[j];
                if (lane == 0) p.fse_new[v] = fpack(start, (uint32_t)nacc);
            } else if (lane == 0) {
                p.ctr->fovf = 1;
            }
            if (lane == 0) c_acc += nacc;
        }
    }
    c_probed = warp_sum(c_probed);
    c_msgs = warp_sum(c_msgs);
    if (p.count_check) {
        c_chk[0] = warp_sum(c_chk[0]);
        c_chk[1] = warp_sum(c_chk[1]);
        if (lane == 0) {
            atomicAdd(&p.ctr->chk_lv, c_chk[0]);
            atomicAdd(&p.ctr->chk_lh, c_chk[1]);
        }
    }
    if (lane == 0) {
        atomicAdd(&p.ctr->arcs, c_arcs);
        atomicAdd(&p.ctr->msgs, c_msgs);
        atomicAdd(&p.ctr->uniq, c_uniq);
        atomicAdd(&p.ctr->staged, c_staged);
        atomicAdd(&p.ctr->probed, c_probed);
        atomicAdd(&p.ctr->accepted, c_acc);
        atomicAdd(&p.ctr->tier[0], c_vert);
        atomicAdd(&p.ctr->prefiltered, c_pref);
    }
}

// Block-per-vertex scalars in shared memory (ints)
enum { SH_UNIQ = 0, SH_OVF = 1, SH_ACC = 2, SH_NC = 3, SH_HI = 4, SH_TMP = 5, SH_START = 6 /* 2 ints */, SH_NEXT = 8,
       SH_WORDS = 48 };

// One block per vertex, any size.  The candidates are processed in passes
// over hub ranges [lo, hi): each pass gathers the messages of its range into
// the shared-memory set (shrinking hi when the set would overflow), checks
// them and appends the survivors to this block's global scratch, copied to
// the new frontier at the end.  L(v) is staged into the shared-memory map when it fits;
// otherwise membership in L(v) is a binary search in its row.
__device__ void gp_block_vertex(const GpParams& p, uint32_t d, int32_t v, uint32_t* S, uint32_t* M, uint32_t* C,
                                uint8_t* B, uint32_t* gacc, int* sh, int* wsum, int* sex, int64_t* sst, int* hist,
                                uint32_t* tv, unsigned long long* cnt) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    const int64_t lb = p.loff[v], ll = p.loff[v + 1] - lb;
    const int64_t nb = p.roff[v], ne = p.roff[v + 1];
    const uint32_t* lv = p.lent + lb;
    const int log_s = p.log_s, S_CAP = 1 << log_s, limit = p.cand_limit;
    int log_m = ceil_log2_i64(2 * ll + 2 * nthr);
    if (log_m < 5) log_m = 5;
    const bool useM = log_m <= p.log_m;
    // L(v) lookups: the shared-memory map, or v's row of the global probe
    // index (a row too long for the map has more than 64 >= kIndexMinLen
    // entries, so it is indexed)
    static_assert(kIndexMinLen <= 64, "rows beyond the block map must be indexed");
    const uint32_t* Mp = M;
    int log_mp = log_m;
    if (!useM) {
        const uint64_t hd = p.hdesc[v];
        Mp = p.htab + (hd >> 8);
        log_mp = (int)(hd & 0xFFu);
    }
    if (useM) {
        for (int s = tid; s < (1 << log_m); s += nthr) M[s] = kEmpty;
        __syncthreads();
        for (int64_t j = tid; j < ll; j += nthr) map_insert(M, log_m, lv[j]);
    }
    if (tid == 0) {
        cnt[0] += ne - nb;
        cnt[3] += ll;
        cnt[6] += 1;
    }
    stage_exact_levels(p.top, v, tv, tid, nthr);
    int64_t total_acc = 0;
    uint32_t lo = 0;
    int64_t width = v;
    uint32_t* hi_sm = reinterpret_cast<uint32_t*>(&sh[SH_HI]);
    // hubs below W (the most frequent messages) are deduplicated in the byte
    // map, in the first pass, for vertices with many messages (for the others
    // clearing and scanning the map costs more than the hashing it saves)
    const uint32_t W = p.rbound[v] >= kByteMinBound ? min((uint32_t)kByteHubs, (uint32_t)v) : 0u;
    const int nbw = (int)((W + 3) / 4);  // byte-map words in use
    for (int q = tid; q < nbw; q += nthr) reinterpret_cast<uint32_t*>(B)[q] = 0u;
    while ((int64_t)lo < (int64_t)v) {
        for (int s = tid; s < S_CAP; s += nthr) S[s] = kEmpty;
        if (tid == 0) {
            sh[SH_UNIQ] = 0;
            sh[SH_OVF] = 0;
            sh[SH_ACC] = 0;
            sh[SH_NC] = 0;
            sh[SH_NEXT] = 0;
            *hi_sm = (uint32_t)min((int64_t)v, (int64_t)lo + width);
        }
        __syncthreads();
        gather_block(p, nb, ne, lo, hi_sm, B, W, S, log_s, useM ? M : nullptr, log_m, limit, &sh[SH_UNIQ],
                     (volatile int*)&sh[SH_OVF], wsum, sex, sst, C, hist, &sh[SH_TMP], cnt[1]);
        __syncthreads();
        const uint32_t hi = *(volatile uint32_t*)hi_sm;
        if (lo < W) {  // first pass: drop L(v)'s hubs from the byte map
            for (int64_t j = tid; j < ll; j += nthr) {
                const uint32_t w = hub_of(lv[j]);
                if (w < W) B[w] = 0;
            }
        }
        // compact the set into C (any order)
        for (int sb = 32 * wid; sb < S_CAP; sb += 32 * nw) {
            const uint32_t h = S[sb + lane];
            const bool has = h != kEmpty;
            const unsigned m = __ballot_sync(kFull, has);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&sh[SH_NC], __popc(m));
            base = __shfl_sync(kFull, base, 0);
            const int idx = base + __popc(m & ((1u << lane) - 1u));
            if (has) {
                if (idx < limit) C[idx] = h;
                else p.ctr->guard = 1;  // invariant broken: report instead of writing out of bounds
            }
        }
        __syncthreads();  // every warp has read the set
        // L(v)'s sorted row in the set's free tail (the byte-map staging below
        // uses its head): the checks' binary searches in L(v) and their side-B
        // scans of it then read shared memory
        const uint32_t* lvp = lv;
        if (ll + (int64_t)nw * kByteStage <= (int64_t)S_CAP) {
            uint32_t* lvs = S + (S_CAP - ll);
            for (int64_t j = tid; j < ll; j += nthr) lvs[j] = lv[j];
            lvp = lvs;
        }
        __syncthreads();
        // entries of L(v) with hub below kTopHubs (the checks' side B starts past them)
        const int lv_top = (int)lower_bound_u32(lvp, ll, pack((uint32_t)kTopHubs, 0));
        const int nc_set = min(*(volatile int*)&sh[SH_NC], limit);  // candidates from the set
        if (tid == 0) cnt[2] += nc_set;
        if (lo < W) {
            // the byte-map candidates: each warp extracts 32 words (up to 128
            // hubs) at a time into its slice of S (free after the compaction;
            // kByteStage words per warp), checks them in full chunks of 32 and
            // carries the remainder; its final remainder (< 32) joins C
            uint32_t* stage = S + wid * kByteStage;
            int f = 0;  // candidates staged
            for (int g = 32 * wid; g < nbw; g += 32 * nw) {
                const uint32_t x = g + lane < nbw ? reinterpret_cast<const uint32_t*>(B)[g + lane] : 0u;
                const uint32_t b4 = (x & 1u) | ((x >> 7) & 2u) | ((x >> 14) & 4u) | ((x >> 21) & 8u);
                const int c = __popc(b4);
                const int incl = warp_incl_scan(c, lane);
                const int tot = __shfl_sync(kFull, incl, 31);
                int o = f + incl - c;
                for (int b = 0; b < 4; ++b)
                    if ((b4 >> b) & 1u) stage[o++] = 4u * (uint32_t)(g + lane) + (uint32_t)b;
                if (lane == 0) cnt[2] += tot;
                f += tot;
                __syncwarp();
                const int nchk = f & ~31;
                for (int cb = 0; cb < nchk; cb += 32) {
                    const uint32_t h = stage[cb + lane];
                    const unsigned okm = check_chunk(p, d, Mp, log_mp, !useM, kBlockSideBMin, kBlockSideBShift, lvp,
                                                     ll, lv_top, h, true, cnt[4], tv, cnt[7], cnt + 8);
                    int base = 0;
                    if (lane == 0 && okm) base = atomicAdd(&sh[SH_ACC], __popc(okm));
                    base = __shfl_sync(kFull, base, 0);
                    if ((okm >> lane) & 1u) gacc[total_acc + base + __popc(okm & ((1u << lane) - 1u))] = h;
                }
                const int rem = f - nchk;
                uint32_t carry = 0u;
                if (lane < rem) carry = stage[nchk + lane];
                __syncwarp();
                if (lane < rem) stage[lane] = carry;
                f = rem;
                __syncwarp();
            }
            int base = 0;
            if (lane == 0 && f) base = atomicAdd(&sh[SH_NC], f);
            base = __shfl_sync(kFull, base, 0);
            if (lane < f) C[base + lane] = stage[lane];  // C holds limit + 32 per warp
            __syncthreads();
        }
        // distance checks of C (the set's candidates, then the byte map's
        // remainders): each warp takes the next chunk of 32 from a shared
        // counter (chunks differ in cost); the survivors are appended
        // (unsorted) to this block's scratch
        const int nc = *(volatile int*)&sh[SH_NC];
        for (;;) {
            int cb = 0;
            if (lane == 0) cb = atomicAdd(&sh[SH_NEXT], 32);
            cb = __shfl_sync(kFull, cb, 0);
            if (cb >= nc) break;
            bool valid = cb + lane < nc;
            const uint32_t h = valid ? C[cb + lane] : 0u;
            // without the map, set candidates may be hubs of v already (they
            // were counted as unique candidates: take them back)
            if (!useM) {
                const bool known = valid && cb + lane < nc_set && map_find(Mp, log_mp, h) != kEmpty;
                const unsigned km = __ballot_sync(kFull, known);
                if (lane == 0) cnt[2] -= __popc(km);
                if (known) valid = false;
            }
            const unsigned okm = check_chunk(p, d, Mp, log_mp, !useM, kBlockSideBMin, kBlockSideBShift, lvp, ll,
                                             lv_top, h, valid, cnt[4], tv, cnt[7], cnt + 8);
            int base = 0;
            if (lane == 0 && okm) base = atomicAdd(&sh[SH_ACC], __popc(okm));
            base = __shfl_sync(kFull, base, 0);
            if ((okm >> lane) & 1u) gacc[total_acc + base + __popc(okm & ((1u << lane) - 1u))] = h;
        }
        __syncthreads();
        total_acc += *(volatile int*)&sh[SH_ACC];
        __syncthreads();
        width = 2 * (int64_t)(hi - lo);
        lo = hi;
    }
    if (total_acc > 0) {
        if (tid == 0) {
            const unsigned long long start = p.ostart ? (unsigned long long)p.ostart[v]
                                                      : atomicAdd(&p.ctr->cursor, (unsigned long long)total_acc);
            *(unsigned long long*)(sh + SH_START) = start;
        }
        __syncthreads();
        const unsigned long long start = *(volatile unsigned long long*)(sh + SH_START);
        if (start + total_acc <= p.fcap) {
            for (int64_t j = tid; j < total_acc; j += nthr) p.fhub_new[start + j] = gacc[j];
            if (tid == 0) {
                p.fse_new[v] = fpack(start, (uint32_t)total_acc);
                if (p.unsorted && total_acc > 1) p.unsorted[atomicAdd(&p.ctr->nU, 1)] = v;  // sorted after the round
            }
        } else if (tid == 0) {
            p.ctr->fovf = 1;
        }
        if (tid == 0) cnt[5] += total_acc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256, 3) k_gp_block(GpParams p) {
    extern __shared__ uint32_t sm[];
    int* sh = reinterpret_cast<int*>(sm);
    int* wsum = sh + SH_WORDS;                                      // 33 ints (+ pad)
    int* hist = wsum + 34;                                          // 256 ints
    uint32_t* tv = reinterpret_cast<uint32_t*>(hist + 256);         // v's exact-distance top-hub masks
    int* sex = reinterpret_cast<int*>(tv + kTopRow);                // blockDim + 1 ints
    int64_t* sst = reinterpret_cast<int64_t*>(sex + ((blockDim.x + 2) & ~1u));  // blockDim int64
    uint32_t* S = reinterpret_cast<uint32_t*>(sst + blockDim.x);
    uint32_t* M = S + (1 << p.log_s);
    uint32_t* C = M + (1 << p.log_m);
    uint8_t* B = reinterpret_cast<uint8_t*>(C + p.cand_limit + (int)blockDim.x);  // kByteHubs bytes
    uint32_t* gacc = p.gscratch + (int64_t)blockIdx.x * p.gscratch_words;
    unsigned long long cnt[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (p.ctr->done) return;
    const uint32_t d = p.ctr->d;
    const int n1 = *p.list_n;
    for (int i = blockIdx.x; i < n1; i += gridDim.x) {
        gp_block_vertex(p, d, p.list[i], S, M, C, B, gacc, sh, wsum, sex, sst, hist, tv, cnt);
        __syncthreads();
    }
    cnt[1] = warp_sum(cnt[1]);
    cnt[4] = warp_sum(cnt[4]);
    if (p.count_check) {
        cnt[8] = warp_sum(cnt[8]);
        cnt[9] = warp_sum(cnt[9]);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&p.ctr->chk_lv, cnt[8]);
            atomicAdd(&p.ctr->chk_lh, cnt[9]);
        }
    }
    if ((threadIdx.x & 31) == 0) {  // lane 0 of each warp holds its warp's unique and prefiltered counts
        atomicAdd(&p.ctr->msgs, cnt[1]);
        atomicAdd(&p.ctr->probed, cnt[4]);
        atomicAdd(&p.ctr->prefiltered, cnt[7]);
        atomicAdd(&p.ctr->uniq, cnt[2]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&p.ctr->arcs, cnt[0]);
        atomicAdd(&p.ctr->staged, cnt[3]);
        atomicAdd(&p.ctr->accepted, cnt[5]);
        atomicAdd(&p.ctr->tier[1], cnt[6]);
    }
}

// Check records of all rows, from the label offsets and the probe index as
// they stand for the coming gather (a finished round returns at once).
__global__ void k_pack_hrec(const int64_t* loff, const uint32_t* lent, const uint64_t* hdesc, uint4* hrec, int64_t n,
                            const RoundCounters* ctr) {
    if (ctr->done) return;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = loff[v], len = loff[v + 1] - a;
        const uint64_t row = hrec_row((uint64_t)a, (uint64_t)len);
        // entries of L(v) with hub < kTopHubs (rows are hub-sorted)
        const uint64_t top = (uint64_t)lower_bound_u32(lent + a, len, pack((uint32_t)kTopHubs, 0));
        const uint64_t hd = hdesc[v] | (top << (32 + kHrecTopShift));
        hrec[v] = make_uint4((uint32_t)row, (uint32_t)(row >> 32), (uint32_t)hd, (uint32_t)(hd >> 32));
    }
}

}  // namespace plb
