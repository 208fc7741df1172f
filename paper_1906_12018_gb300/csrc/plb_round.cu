// Round kernels of the vertex-centric labeling (Alg. 3, Sec. 3.1).
// See plb_kernels.cuh for the per-round pipeline.
#include "plb_kernels.cuh"
#include "plb_round.cuh"

namespace plb {

namespace {

constexpr int kTileItems = 2048;  // items per block tile in flat (load-balanced) kernels

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// First and last row of offsets off[0..nrows] that intersect items [p0, p1).
__device__ __forceinline__ void tile_rows(const int64_t* off, int64_t nrows, int64_t p0, int64_t p1,
                                          int64_t* r0, int64_t* r1) {
    *r0 = row_of(off, 0, nrows - 1, p0);
    *r1 = row_of(off, 0, nrows - 1, p1 - 1);
}

}  // namespace

// ------------------------------------------------------------ validation
__global__ void k_check_rowptr(const int64_t* row_ptr, int64_t n, int64_t nnz, int* err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = row_ptr[i];
        bool bad = x < 0 || x > nnz;
        if (i == 0 && x != 0) bad = true;
        if (i == n && x != nnz) bad = true;
        if (i < n && row_ptr[i + 1] < x) bad = true;
        if (bad) atomicOr(err, 1);
    }
}

// Per arc (u -> c): 0 <= c < n, c != u, rows strictly ascending, and the
// reverse arc (c -> u) exists (binary search in row c).
__global__ void k_check_cols(const int64_t* row_ptr, const int32_t* col, int64_t n, int64_t nnz, int* err) {
    __shared__ int64_t sh_r[2];
    const int64_t ntiles = (nnz + kTileItems - 1) / kTileItems;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(nnz, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(row_ptr, n, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int64_t u = row_of(row_ptr, r0, r1, p);
            const int32_t c = col[p];
            bool bad = c < 0 || (int64_t)c >= n || (int64_t)c == u;
            if (!bad && p > row_ptr[u] && col[p - 1] >= c) bad = true;
            if (!bad) {
                const int64_t b = row_ptr[c], e = row_ptr[c + 1];
                int64_t lo = b, hi = e;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if ((int64_t)col[mid] < u) lo = mid + 1; else hi = mid;
                }
                if (lo >= e || (int64_t)col[lo] != u) bad = true;
            }
            if (bad) atomicOr(err, 2);
        }
    }
}

__global__ void k_check_order(const int32_t* order, int64_t n, int* seen, int* err) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t id = order[r];
        if (id < 0 || (int64_t)id >= n) {
            atomicOr(err, 4);
        } else if (atomicAdd(seen + id, 1) != 0) {
            atomicOr(err, 4);
        }
    }
}

// ------------------------------------------------------------ relabel
__global__ void k_inverse(const int32_t* order, int32_t* inv, int64_t n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        inv[order[r]] = (int32_t)r;
}

__global__ void k_rank_degree(const int64_t* row_ptr, const int32_t* order, int64_t* rdeg, int64_t n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t id = order[r];
        rdeg[r] = row_ptr[id + 1] - row_ptr[id];
    }
}

// rcol[roff[r] + j] = rank of the j-th neighbour of order[r] (row order kept).
__global__ void k_relabel(const int64_t* row_ptr, const int32_t* col, const int32_t* order, const int32_t* inv,
                          const int64_t* roff, int32_t* rcol, int64_t n, int64_t nnz) {
    __shared__ int64_t sh_r[2];
    const int64_t ntiles = (nnz + kTileItems - 1) / kTileItems;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(nnz, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(roff, n, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int64_t r = row_of(roff, r0, r1, p);
            const int32_t id = order[r];
            rcol[p] = inv[col[row_ptr[id] + (p - roff[r])]];
        }
    }
}

// L(v) = dL(v) = {(v, 0)}; active = vertices with at least one neighbour.
__global__ void k_init(const int64_t* roff, int64_t n, int64_t* loff, uint32_t* lent, uint64_t* fse,
                       uint32_t* fhub, int32_t* A, RoundCounters* ctr) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        loff[v] = v;
        lent[v] = pack((uint32_t)v, 0);
        fhub[v] = (uint32_t)v;
        fse[v] = fpack((uint64_t)v, 1);
        const bool act = roff[v + 1] > roff[v];
        const unsigned am = __activemask();
        const unsigned m = __ballot_sync(am, act);
        if (m) {
            const int leader = __ffs(m) - 1;
            int base = 0;
            if (lane_id() == leader) base = atomicAdd(&ctr->nA, __popc(m));
            base = __shfl_sync(am, base, leader);
            if (act) A[base + __popc(m & ((1u << lane_id()) - 1u))] = (int32_t)v;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) loff[n] = n;
}

// ------------------------------------------------------------ frontier
// adeg[i] = degree of active vertex A[i] (0 beyond nA), for the flat mark.
__global__ void k_active_degree(const int64_t* roff, const int32_t* A, const RoundCounters* ctr, int64_t* adeg,
                                int64_t n) {
    if (ctr->done) return;
    const int nA = ctr->nA;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = 0;
        if (i < nA) {
            const int32_t a = A[i];
            x = roff[a + 1] - roff[a];
        }
        adeg[i] = x;
    }
}

// Flat over the arcs of the active list: v in N(a) receives when min dL(a) < v
// (some new hub of a outranks v); recv[v] accumulates |dL(a)| over such
// neighbours, an upper bound on v's messages.
__global__ void k_mark(const int64_t* roff, const int32_t* rcol, const uint64_t* fse, const uint32_t* fhub,
                       const int32_t* A, const int64_t* aoff, const RoundCounters* ctr, unsigned long long* recv,
                       int64_t n) {
    __shared__ int64_t sh_r[2];
    if (ctr->done) return;
    const int64_t nA = ctr->nA;
    if (nA == 0) return;
    const int64_t total = aoff[n];
    const int64_t ntiles = (total + kTileItems - 1) / kTileItems;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(total, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(aoff, nA, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int64_t i = row_of(aoff, r0, r1, p);
            const int32_t a = A[i];
            const uint64_t f = fse[a];
            const uint32_t minh = fhub[fstart(f)];
            const int32_t v = rcol[roff[a] + (p - aoff[i])];
            if ((uint32_t)v > minh) atomicAdd(recv + v, (unsigned long long)fcount(f));
        }
    }
}

// Receivers (recv[v] > 0) are routed by the candidate bound min(v, recv[v]),
// |L(v)| and degree: warp tier (R) or block tier (O1); the bound is kept in
// rbound[v] (it sizes the warp tier's tables).  Also clears recv and the new
// frontier descriptors, and sums the bounds.
__global__ void k_collect(unsigned long long* recv, const int64_t* roff, const int64_t* loff, int64_t n,
                          uint64_t* fse_new, int32_t* R, int32_t* O1, uint32_t* rbound, RoundCounters* ctr,
                          TierLimits lim) {
    if (ctr->done) return;
    unsigned long long bsum = 0;
    const int lane = lane_id();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        fse_new[v] = 0;
        const unsigned long long c = recv[v];
        int tier = -1;
        if (c) {
            recv[v] = 0;
            const unsigned long long bound = c < (unsigned long long)v ? c : (unsigned long long)v;
            bsum += bound;
            rbound[v] = (uint32_t)bound;  // v < 2^24
            const int64_t ll = loff[v + 1] - loff[v];
            const int64_t deg = roff[v + 1] - roff[v];
            tier = ((int64_t)bound <= lim.warp_bound && ll <= lim.warp_label && deg <= lim.warp_deg) ? 0 : 1;
        }
        const unsigned am = __activemask();
        int32_t* lists[2] = {R, O1};
        int* counts[2] = {&ctr->nR, &ctr->nO1};
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const unsigned m = __ballot_sync(am, tier == t);
            if (m) {
                const int leader = __ffs(m) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(counts[t], __popc(m));
                base = __shfl_sync(am, base, leader);
                if (tier == t) lists[t][base + __popc(m & ((1u << lane) - 1u))] = (int32_t)v;
            }
        }
    }
    bsum = warp_sum(bsum);
    if (lane == 0 && bsum) atomicAdd(&ctr->bound_sum, bsum);
}

__global__ void k_after_collect(RoundCounters* ctr) {
    if (ctr->done) return;
    ctr->nO1_base = ctr->nO1;
    ctr->nO2_base = ctr->nO2;
    ctr->nA_saved = ctr->nA;
    ctr->nA = 0;
}

// Round 1 (Alg. 3 with d = 1).  The candidates of v are its neighbours a < v
// (each sends its only label (a, 0)), they are distinct, and none is pruned:
// a witness w of (a, 1) at v would need d(w, v) + d(w, a) <= 1 with w in
// L(v) = {(v, 0)} and in L(a) = {(a, 0)}, impossible for a != v.  So
// dL_1(v) = {a in N(v) : a < v}: one warp per vertex appends it (unsorted;
// the merge step sorts the rows), clears the other frontier descriptors and
// restarts the active list.  Counted like the general round: one message,
// one unique candidate and one accepted label per such neighbour.
__global__ void k_round1(const int64_t* roff, const int32_t* rcol, int64_t n, uint64_t* fse_new, uint32_t* fhub_new,
                         unsigned long long fcap, RoundCounters* ctr) {
    if (ctr->done) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->nA_saved = ctr->nA;
        ctr->nA = 0;
    }
    const int lane = lane_id();
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long c_acc = 0, c_arcs = 0, c_recv = 0;
    for (int64_t v = warp0; v < n; v += nwarps) {
        const int64_t nb = roff[v], ne = roff[v + 1];
        int c = 0;
        for (int64_t j0 = nb; j0 < ne; j0 += 128) {  // four independent loads per lane
            int k = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t j = j0 + 32 * u + lane;
                k += (j < ne && rcol[j] < v) ? 1 : 0;
            }
            c += k;
        }
        c = warp_sum(c);
        if (c == 0) {
            if (lane == 0) fse_new[v] = 0;
            continue;
        }
        unsigned long long start = 0;
        if (lane == 0) start = atomicAdd(&ctr->cursor, (unsigned long long)c);
        start = __shfl_sync(kFull, start, 0);
        if (start + c > fcap) {  // cannot happen: the buffer holds every arc
            if (lane == 0) {
                ctr->fovf = 1;
                fse_new[v] = 0;
            }
            continue;
        }
        int o = 0;
        for (int64_t j0 = nb; j0 < ne; j0 += 32) {
            const int64_t j = j0 + lane;
            const int32_t a = j < ne ? rcol[j] : INT32_MAX;
            const bool up = a < v;
            const unsigned m = __ballot_sync(kFull, up);
            if (up) fhub_new[start + o + __popc(m & ((1u << lane) - 1u))] = (uint32_t)a;
            o += __popc(m);
        }
        if (lane == 0) {
            fse_new[v] = fpack(start, (uint32_t)c);
            c_acc += c;
            c_arcs += ne - nb;
            c_recv += 1;
        }
    }
    if (lane == 0 && c_recv) {
        atomicAdd(&ctr->accepted, c_acc);
        atomicAdd(&ctr->msgs, c_acc);
        atomicAdd(&ctr->uniq, c_acc);
        atomicAdd(&ctr->arcs, c_arcs);
        atomicAdd(&ctr->tier[0], c_recv);
        atomicAdd(&ctr->nR, (int)c_recv);
    }
}

// Reset before re-running the gather/prune of a round with a bigger buffer.
__global__ void k_rerun_reset(RoundCounters* ctr, uint64_t* fse_new, int64_t n) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        fse_new[v] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->nO1 = ctr->nO1_base;
        ctr->nO2 = ctr->nO2_base;
        ctr->cursor = 0;
        ctr->accepted = 0;
        ctr->fovf = 0;
        ctr->arcs = ctr->msgs = ctr->uniq = ctr->staged = ctr->probed = 0;
        ctr->tier[0] = ctr->tier[1] = ctr->tier[2] = 0;
    }
}

// ------------------------------------------------------- gather + prune
constexpr int kPrefilterMinItems = 12;  // prefilter only candidates with longer checks
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
            const uint4 a = cj[0], b = cj[1];
            const uint32_t* e = ev + (i - 1) * kTopWords;
            hit |= (a.x & e[0]) | (a.y & e[1]) | (a.z & e[2]) | (a.w & e[3]) | (b.x & e[4]) | (b.y & e[5]) |
                   (b.z & e[6]) | (b.w & e[7]);
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
// witness.  Returns the lanes whose candidate survives.
__device__ __forceinline__ unsigned check_chunk(const GpParams& p, uint32_t d, const uint32_t* M, int log_m,
                                                bool mv_global, int b_min, int b_shift, const uint32_t* lv,
                                                int64_t lvlen, uint32_t h, bool valid, unsigned* pm_sm,
                                                unsigned long long& probed, const uint32_t* tv,
                                                unsigned long long& prefiltered) {
    const int lane = threadIdx.x & 31;
    int64_t base = 0;  // A: start of L(h); B: start of h's probe table
    int items = 0, meta = 0;  // meta: 0 = side A, else log2(table size) + 1
    if (valid) {
        const int64_t hb = p.loff[h];
        const int la = (int)(p.loff[h + 1] - hb) - 1;
        base = hb;
        items = la;
        if (la >= b_min) {
            const int64_t x0 = p.hoff[h], x1 = p.hoff[h + 1];
            if (x1 > x0) {
                const int lb = (int)lower_bound_u32(lv, lvlen, pack(h, 0));
                if (mv_global ? lb < la : (lb << b_shift) < la) {
                    items = lb;
                    base = x0;
                    meta = __ffs((int)(x1 - x0));  // log2 + 1
                }
            }
        }
    }
    // candidates with a long check first try the top-hub prefilter
    const unsigned pf = top_prefilter(p.top, tv, d, h, valid && items >= kPrefilterMinItems);
    if (lane == 0) prefiltered += __popc(pf);
    if ((pf >> lane) & 1u) {
        valid = false;
        items = 0;
    }
    const unsigned vmask = __ballot_sync(kFull, valid);
    if (lane == 0) *pm_sm = 0;
    const int incl = warp_incl_scan(items, lane);
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - items;
    __syncwarp();
    for (int ib = 0; ib < total; ib += 32) {
        const unsigned pm = *(volatile unsigned*)pm_sm;
        if ((pm & vmask) == vmask) break;
        const int it = ib + lane;
        const int k = warp_owner(excl, it);
        const int64_t bk = __shfl_sync(kFull, base, k);
        const int exk = __shfl_sync(kFull, excl, k);
        const int mk = __shfl_sync(kFull, meta, k);
        if (it < total && !((pm >> k) & 1u)) {
            const int j = it - exk;
            bool hit = false;
            if (mk == 0) {
                const uint32_t x = p.lent[bk + j];
                const uint32_t dv = map_find(M, log_m, hub_of(x));
                hit = dv != kEmpty && dv + dist_of(x) <= d;
            } else {
                const uint32_t y = lv[j];
                const uint32_t dh = map_find(p.htab + bk, mk - 1, hub_of(y));
                hit = dh != kEmpty && dh + dist_of(y) <= d;
            }
            ++probed;
            if (hit) atomicOr(pm_sm, 1u << k);
        }
        __syncwarp();
    }
    const unsigned pm = *(volatile unsigned*)pm_sm;
    __syncwarp();
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
                // the hubs of dL_{d-1}(a) are <= a (a itself only for d = 1):
                // for a < hi the whole row lies below hi
                const uint32_t* row = p.fhub + fstart(f);
                const int64_t a0 = lo ? lower_bound_u32(row, n0, lo) : 0;
                const int64_t a1 = (uint32_t)a < hi ? (int64_t)n0 : lower_bound_u32(row, n0, hi);
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
#pragma unroll
            for (int u = 0; u < kGatherUnroll; ++u) {
                const int it = ib + 32 * u + lane;
                const int k = warp_owner(excl, it);
                const int64_t stk = __shfl_sync(kFull, st, k);
                const int exk = __shfl_sync(kFull, excl, k);
                hv[u] = it < total ? p.fhub[stk + (it - exk)] : kEmpty;
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
// `limit`, its range (hubs >= W) is shrunk (shrink_pass) and the current tile
// redone, so messages gathered below the new bound are kept.
__device__ void gather_block(const GpParams& p, int64_t nb, int64_t ne, uint32_t lo, uint32_t* hi_sm, uint8_t* B,
                             uint32_t W, uint32_t* S, int log_s, const uint32_t* M, int log_m, int limit, int* cnt_sm,
                             volatile int* ovf_sm, int* wsum, int* sex, int64_t* sst, uint32_t* C, int* hist, int* tmp,
                             unsigned long long& msgs) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int64_t t0 = nb; t0 < ne;) {
        const uint32_t hi = *(volatile uint32_t*)hi_sm;
        const int64_t j = t0 + tid;
        int c = 0;
        int64_t st = 0;
        if (j < ne) {
            const int32_t a = p.rcol[j];
            const uint64_t f = p.fse[a];
            const uint32_t n0 = fcount(f);
            if (n0) {
                // the hubs of dL_{d-1}(a) are <= a (a itself only for d = 1):
                // for a < hi the whole row lies below hi
                const uint32_t* row = p.fhub + fstart(f);
                const int64_t a0 = lo ? lower_bound_u32(row, n0, lo) : 0;
                const int64_t a1 = (uint32_t)a < hi ? (int64_t)n0 : lower_bound_u32(row, n0, hi);
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
        const int nw = nthr >> 5, lane = tid & 31;
        const int per_w = (((total + nw - 1) / nw) + 31) & ~31;
        const int wbeg = (tid >> 5) * per_w, wend = min(total, wbeg + per_w);
        if (wbeg < wend) {
            int k0 = 0, hk = nne - 1;  // row of wbeg: largest k with sex[k] <= wbeg
            while (k0 < hk) {
                const int mid = (k0 + hk + 1) >> 1;
                if (sex[mid] <= wbeg) k0 = mid; else hk = mid - 1;
            }
            bool stop = false;
            for (int it0 = wbeg; it0 < wend && !stop; k0 += 32) {
                const int kr = k0 + lane;
                const int ex = kr < nne ? sex[kr] : total;
                const int64_t stv = kr < nne ? sst[kr] : 0;
                const int wcap = k0 + 32 < nne ? sex[k0 + 32] : total;
                const int wend_w = min(wend, wcap);
                for (int ib = it0; ib < wend_w; ib += 32 * kGatherUnroll) {
                    uint32_t hv[kGatherUnroll];
#pragma unroll
                    for (int u = 0; u < kGatherUnroll; ++u) {
                        const int it = ib + 32 * u + lane;
                        const int kk = warp_owner(ex, it);
                        const int exk = __shfl_sync(kFull, ex, kk);
                        const int64_t stk = __shfl_sync(kFull, stv, kk);
                        hv[u] = it < wend_w ? p.fhub[stk + (it - exk)] : kEmpty;
                    }
                    int nins = 0;
#pragma unroll
                    for (int u = 0; u < kGatherUnroll; ++u) {
                        const uint32_t h = hv[u];
                        if (h < W) {
                            B[h] = 1;
                        } else if (h != kEmpty && (!M || map_find(M, log_m, h) == kEmpty)) {
                            if (*(volatile int*)cnt_sm >= limit) *ovf_sm = 1;
                            else nins += set_insert(S, log_s, h) ? 1 : 0;
                        }
                    }
                    nins = warp_sum(nins);
                    if (lane == 0 && nins) atomicAdd(cnt_sm, nins);
                    if (__any_sync(kFull, *ovf_sm != 0)) {
                        stop = true;
                        break;
                    }
                }
                it0 = wend_w;
            }
        }
        if (tid == 0) msgs += total;
        __syncthreads();
        // concurrent inserts can pass the limit without raising the flag
        if (*ovf_sm || *(volatile int*)cnt_sm > limit) {
            shrink_pass(S, log_s, C, limit, lo > W ? lo : W, hi_sm, cnt_sm, hist, tmp);  // S holds hubs >= W
            if (tid == 0) *ovf_sm = 0;
            __syncthreads();
            continue;  // redo this tile with the smaller range
        }
        t0 += nthr;
    }
}

// One warp per vertex (tables in shared memory):
//  1. stage L(v) into the hub-keyed map M;
//  2. gather the unique messages into the set S;
//  3. compact S in place and check the candidates 32 at a time;
//  4. append the accepted hubs (unsorted) to the new frontier.
// A vertex whose unique candidates exceed cand_limit goes to the block tier.
__global__ void __launch_bounds__(256, 3) k_gp_warp(GpParams p) {
    extern __shared__ uint32_t sm[];
    const int lane = lane_id(), wib = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int S_CAP = 1 << p.log_s, M_CAP = 1 << p.log_m;
    int* wsc = reinterpret_cast<int*>(sm) + wib * 4;  // [0] unique count [1] overflow [3] pruned mask
    uint32_t* tvs = sm + 4 * nwarps;                   // per warp: v's exact-distance top-hub masks
    uint32_t* S = tvs + nwarps * kTopRow + wib * (S_CAP + M_CAP);
    uint32_t* M = S + S_CAP;
    unsigned long long c_arcs = 0, c_msgs = 0, c_uniq = 0, c_staged = 0, c_probed = 0, c_acc = 0, c_vert = 0;
    unsigned long long c_pref = 0;
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
        const int log_m = max(5, ceil_log2_i64(2 * ll));
        for (int s = lane; s < (1 << log_s); s += 32) S[s] = kEmpty;
        for (int s = lane; s < (1 << log_m); s += 32) M[s] = kEmpty;
        if (lane == 0) {
            wsc[0] = 0;
            wsc[1] = 0;
        }
        __syncwarp();
        for (int64_t j = lane; j < ll; j += 32) map_insert(M, log_m, p.lent[lb + j]);
        __syncwarp();
        const int64_t nb = p.roff[v], ne = p.roff[v + 1];
        const bool ok = gather_range(p, nb, ne, 32, 0u, (uint32_t)v, S, log_s, M, log_m, p.cand_limit, &wsc[0],
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
            c_staged += ll;
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
        // distance checks, 32 candidates at a time; survivors compacted in place
        uint32_t* tv = tvs + wib * kTopRow;
        if (nc > 0) stage_exact_levels(p.top, v, tv, lane, 32);
        __syncwarp();
        int nacc = 0;
        for (int cb = 0; cb < nc; cb += 32) {
            const bool valid = cb + lane < nc;
            const uint32_t h = valid ? S[cb + lane] : 0u;
            __syncwarp();
            const unsigned okm = check_chunk(p, d, M, log_m, false, kWarpSideBMin, kWarpSideBShift, p.lent + lb, ll, h,
                                             valid, (unsigned*)&wsc[3],
                                             c_probed, tv, c_pref);
            if ((okm >> lane) & 1u) S[nacc + __popc(okm & ((1u << lane) - 1u))] = h;
            nacc += __popc(okm);
            __syncwarp();
        }
        if (nacc > 0) {
            unsigned long long start = 0;
            if (lane == 0) start = atomicAdd(&p.ctr->cursor, (unsigned long long)nacc);
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
enum { SH_UNIQ = 0, SH_OVF = 1, SH_ACC = 2, SH_NC = 3, SH_HI = 4, SH_TMP = 5, SH_START = 6 /* 2 ints */,
       SH_PM = 16 /* one word per warp */, SH_WORDS = 48 };

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
        const int64_t x0 = p.hoff[v], x1 = p.hoff[v + 1];
        Mp = p.htab + x0;
        log_mp = __ffsll((unsigned long long)(x1 - x0)) - 1;
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
    const uint32_t W = p.rbound[v] >= (uint32_t)(kByteHubs / 4) ? min((uint32_t)kByteHubs, (uint32_t)v) : 0u;
    const int nbw = (int)((W + 3) / 4);  // byte-map words in use
    for (int q = tid; q < nbw; q += nthr) reinterpret_cast<uint32_t*>(B)[q] = 0u;
    while ((int64_t)lo < (int64_t)v) {
        for (int s = tid; s < S_CAP; s += nthr) S[s] = kEmpty;
        if (tid == 0) {
            sh[SH_UNIQ] = 0;
            sh[SH_OVF] = 0;
            sh[SH_ACC] = 0;
            sh[SH_NC] = 0;
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
        __syncthreads();
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
                    const unsigned okm = check_chunk(p, d, Mp, log_mp, !useM, kBlockSideBMin, kBlockSideBShift, lv,
                                                     ll, h, true,
                                                     (unsigned*)&sh[SH_PM + wid], cnt[4], tv, cnt[7]);
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
        // remainders): warp w takes candidate chunks w, w + nw, ...; the
        // survivors are appended (unsorted) to this block's scratch
        const int nc = *(volatile int*)&sh[SH_NC];
        for (int cb = 32 * wid; cb < nc; cb += 32 * nw) {
            bool valid = cb + lane < nc;
            const uint32_t h = valid ? C[cb + lane] : 0u;
            // without the map, set candidates may be hubs of v already
            if (!useM && valid && cb + lane < nc_set && map_find(Mp, log_mp, h) != kEmpty) valid = false;
            const unsigned okm = check_chunk(p, d, Mp, log_mp, !useM, kBlockSideBMin, kBlockSideBShift, lv, ll, h,
                                             valid, (unsigned*)&sh[SH_PM + wid],
                                             cnt[4], tv, cnt[7]);
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
            const unsigned long long start = atomicAdd(&p.ctr->cursor, (unsigned long long)total_acc);
            *(unsigned long long*)(sh + SH_START) = start;
        }
        __syncthreads();
        const unsigned long long start = *(volatile unsigned long long*)(sh + SH_START);
        if (start + total_acc <= p.fcap) {
            for (int64_t j = tid; j < total_acc; j += nthr) p.fhub_new[start + j] = gacc[j];
            if (tid == 0) p.fse_new[v] = fpack(start, (uint32_t)total_acc);
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
    unsigned long long cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (p.ctr->done) return;
    const uint32_t d = p.ctr->d;
    const int n1 = *p.list_n;
    for (int i = blockIdx.x; i < n1; i += gridDim.x) {
        gp_block_vertex(p, d, p.list[i], S, M, C, B, gacc, sh, wsum, sex, sst, hist, tv, cnt);
        __syncthreads();
    }
    cnt[1] = warp_sum(cnt[1]);
    cnt[4] = warp_sum(cnt[4]);
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

// ------------------------------------------------------------ probe index
// Table size of row x: 2^ceil(log2(2|L(x)|)) for rows of >= kIndexMinLen
// entries, else 0 (those rows are always scanned, never probed).
__global__ void k_index_size(const int64_t* loff, int64_t n, int64_t* hsz, const RoundCounters* ctr) {
    if (ctr->done) return;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = loff[x + 1] - loff[x];
        hsz[x] = l >= kIndexMinLen ? (int64_t(1) << ceil_log2_i64(2 * l)) : 0;
    }
}

// htab[0 .. hoff[n]) = kEmpty (size read on the device).
__global__ void k_index_clear(uint32_t* htab, const int64_t* hoff_n) {
    const int64_t total = *hoff_n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        htab[i] = kEmpty;
}

// Insert every entry of an indexed row into its table (tables pre-filled
// with kEmpty): flat over entries.
__global__ void k_index_fill(const int64_t* loff, const uint32_t* lent, const int64_t* hoff, uint32_t* htab,
                             int64_t n) {
    __shared__ int64_t sh_r[2];
    const int64_t total = loff[n];
    const int64_t ntiles = (total + kTileItems - 1) / kTileItems;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(total, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(loff, n, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        for (int64_t q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
            const int64_t x = row_of(loff, r0, r1, q);
            const int64_t b = hoff[x], sz = hoff[x + 1] - b;
            if (sz > 0) map_insert(htab + b, __ffs((int)sz) - 1, lent[q]);
        }
    }
}

// One warp per indexed row: the table is built in shared memory (rows whose
// table has up to kIndexSmemSlots slots) and written out whole, empty slots
// included; larger tables are cleared and filled in place with atomics.
constexpr int kIndexWarps = 8;
constexpr int kIndexSmemSlots = 2048;

__global__ void __launch_bounds__(kIndexWarps * 32) k_index_build(const int64_t* loff, const uint32_t* lent,
                                                                  const int64_t* hoff, uint32_t* htab, int64_t n,
                                                                  const RoundCounters* ctr) {
    extern __shared__ uint32_t ibuf[];
    if (ctr->done) return;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    uint32_t* buf = ibuf + w * kIndexSmemSlots;
    const int64_t nwarps = (int64_t)gridDim.x * kIndexWarps;
    for (int64_t base = ((int64_t)blockIdx.x * kIndexWarps + w) * 32; base < n; base += nwarps * 32) {
        const int64_t x = base + lane;
        int64_t hb = 0, P = 0;
        if (x < n) {
            hb = hoff[x];
            P = hoff[x + 1] - hb;
        }
        unsigned m = __ballot_sync(kFull, P > 0);
        while (m) {
            const int k = __ffs(m) - 1;
            m &= m - 1;
            const int64_t xk = base + k;
            const int64_t hbk = __shfl_sync(kFull, hb, k);
            const int Pk = (int)__shfl_sync(kFull, P, k);
            const int lg = __ffs(Pk) - 1;
            const int64_t lb = loff[xk], ll = loff[xk + 1] - lb;
            uint32_t* tab = Pk <= kIndexSmemSlots ? buf : htab + hbk;
            for (int sl = lane; sl < Pk; sl += 32) tab[sl] = kEmpty;
            __syncwarp();
            for (int64_t j = lane; j < ll; j += 32) map_insert(tab, lg, lent[lb + j]);
            __syncwarp();
            if (Pk <= kIndexSmemSlots) {
                for (int sl = lane; sl < Pk; sl += 32) htab[hbk + sl] = buf[sl];
                __syncwarp();
            }
        }
    }
}

// ------------------------------------------------------------ merge
// next active list + per-vertex new row lengths
__global__ void k_next_active(const int64_t* loff, const uint64_t* fse_new, int64_t n, int64_t* newlen, int32_t* A,
                              RoundCounters* ctr) {
    if (ctr->done) return;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = fcount(fse_new[v]);
        newlen[v] = (loff[v + 1] - loff[v]) + c;
        const bool act = c > 0;
        const unsigned am = __activemask();
        const unsigned m = __ballot_sync(am, act);
        if (m) {
            const int leader = __ffs(m) - 1;
            int base = 0;
            if (lane_id() == leader) base = atomicAdd(&ctr->nA, __popc(m));
            base = __shfl_sync(am, base, leader);
            if (act) A[base + __popc(m & ((1u << lane_id()) - 1u))] = (int32_t)v;
        }
    }
}

// ------------------------------------------------- sort new frontier rows
// The gather/prune kernels append each vertex's accepted hubs unsorted; one
// warp per active vertex sorts its row: up to 32 entries in registers (a
// bitonic network over the lanes), up to kWarpSortMax in shared memory;
// longer rows are listed for k_sort_rows_block.
constexpr int kWarpSortMax = 1024;
constexpr int kSortWarps = 8;
constexpr int kBlockSortSmem = 16384;

__global__ void __launch_bounds__(kSortWarps * 32) k_sort_rows_warp(const uint64_t* fse_new, uint32_t* fhub_new,
                                                                   const int32_t* A, RoundCounters* ctr,
                                                                   int32_t* big, int32_t* giant) {
    __shared__ uint32_t buf[kSortWarps][kWarpSortMax];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    if (ctr->done) return;
    const int nA = ctr->nA;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nA; i += nw) {
        const int32_t v = A[i];
        const uint64_t f = fse_new[v];
        const int c = (int)fcount(f);
        uint32_t* row = fhub_new + fstart(f);
        if (c <= 1) continue;
        if (c <= 32) {
            uint32_t x = lane < c ? row[lane] : kEmpty;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const uint32_t y = __shfl_xor_sync(kFull, x, j);
                    const bool up = (lane & k) == 0, lower = (lane & j) == 0;
                    x = (lower == up) ? min(x, y) : max(x, y);
                }
            }
            if (lane < c) row[lane] = x;
        } else if (c <= kWarpSortMax) {
            int P = 64;
            while (P < c) P <<= 1;
            uint32_t* b = buf[w];
            for (int j = lane; j < P; j += 32) b[j] = j < c ? row[j] : kEmpty;
            __syncwarp();
            group_bitonic_sort(b, P, lane, 32, WarpSync());
            for (int j = lane; j < c; j += 32) row[j] = b[j];
            __syncwarp();
        } else if (lane == 0) {
            if (c <= kBlockSortSmem) big[atomicAdd(&ctr->nBig, 1)] = v;
            else giant[atomicAdd(&ctr->nGiant, 1)] = v;
        }
    }
}

// One block per long row: bitonic sort in a power-of-two buffer (shared
// memory for rows up to kBlockSortSmem entries; longer rows use this block's
// global scratch).  Launched once for each list.

__global__ void __launch_bounds__(1024) k_sort_rows_block(const uint64_t* fse_new, uint32_t* fhub_new,
                                                          const int32_t* big, const int* nbig,
                                                          uint32_t* scratch, int64_t scratch_words,
                                                          const RoundCounters* ctr) {
    extern __shared__ uint32_t sbuf[];
    if (ctr->done) return;
    const int nBig = *nbig;
    for (int i = blockIdx.x; i < nBig; i += gridDim.x) {
        const uint64_t f = fse_new[big[i]];
        const int64_t c = fcount(f);
        uint32_t* row = fhub_new + fstart(f);
        int64_t P = 1;
        while (P < c) P <<= 1;
        uint32_t* b = P <= kBlockSortSmem ? sbuf : scratch + (int64_t)blockIdx.x * scratch_words;
        for (int64_t j = threadIdx.x; j < P; j += blockDim.x) b[j] = j < c ? row[j] : kEmpty;
        __syncthreads();
        group_bitonic_sort(b, (int)P, threadIdx.x, blockDim.x, BlockSync());
        for (int64_t j = threadIdx.x; j < c; j += blockDim.x) row[j] = b[j];
        __syncthreads();
    }
}

// Old entries move to their place in the merged row: flat over old entries.
__global__ void k_merge_old(const int64_t* loff, const uint32_t* lent, const int64_t* loff_new, uint32_t* lent_new,
                            const uint64_t* fse_new, const uint32_t* fhub_new, int64_t n, const RoundCounters* ctr) {
    __shared__ int64_t sh_r[2];
    if (ctr->done) return;
    const int64_t total = loff[n];
    const int64_t ntiles = (total + kTileItems - 1) / kTileItems;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(total, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(loff, n, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        for (int64_t q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
            const int64_t v = row_of(loff, r0, r1, q);
            const uint32_t e = lent[q];
            const uint64_t f = fse_new[v];
            int64_t pos = loff_new[v] + (q - loff[v]);
            const uint32_t c = fcount(f);
            if (c) pos += lower_bound_u32(fhub_new + fstart(f), c, hub_of(e));
            lent_new[pos] = e;
        }
    }
}

// New entries (dist d) of each active vertex: warp per vertex.
__global__ void k_merge_new(const int64_t* loff, const uint32_t* lent, const int64_t* loff_new, uint32_t* lent_new,
                            const uint64_t* fse_new, const uint32_t* fhub_new, const int32_t* A,
                            const RoundCounters* ctr, uint32_t* top) {
    if (ctr->done) return;
    const uint32_t d = ctr->d;
    const int nA = ctr->nA;
    const int lane = lane_id();
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nA; i += nw) {
        const int32_t v = A[i];
        const uint64_t f = fse_new[v];
        const uint32_t c = fcount(f);
        const uint32_t* fr = fhub_new + fstart(f);
        const int64_t ob = loff[v], ol = loff[v + 1] - ob;
        for (uint32_t j = lane; j < c; j += 32) {
            const uint32_t h = fr[j];
            const int64_t pos = loff_new[v] + j + lower_bound_u32(lent + ob, ol, pack(h, 0));
            lent_new[pos] = pack(h, d);
            if (h < (uint32_t)kTopHubs && d <= (uint32_t)kTopLevels) {
                uint32_t* tv = top + (int64_t)v * kTopRow + (h >> 5);
                for (int t = (int)d; t <= kTopLevels; ++t) atomicOr(tv + (t - 1) * kTopWords, 1u << (h & 31));
            }
        }
    }
}

// Masks start empty (distance-0 self labels are not part of any level).
__global__ void k_top_init(uint32_t* top, int64_t n) {
    const int64_t words = n * kTopRow;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
        top[i] = 0u;
}


// ------------------------------------------------------------ loop control
// Host-driven rounds: set the round number.
__global__ void k_set_round(RoundCounters* ctr, uint32_t d) { ctr->d = d; }

// Graph-driven rounds (one thread each).
// Begin: next round number.
__global__ void k_g_begin(RoundCounters* ctr) {
    if (ctr->done) return;
    ctr->d += 1;
}

// After the frontier step: stop before the gather when the round's candidate
// bound (an upper bound on its new-frontier entries) exceeds the buffer of
// parity x.
__global__ void k_g_bound(RoundCounters* ctr, int x) {
    if (ctr->done) return;
    if ((long long)ctr->bound_sum > ctr->fcap[x]) {
        ctr->fallback = kStopBeforeGather;
        ctr->done = 1;
    }
}

// After the gather/prune kernels: stop on a capacity problem (resume on the
// host), on an empty round (finished) or on a distance above 254; else
// account the new labels and record the round's statistics.
__global__ void k_g_check(RoundCounters* ctr, RoundStat* stats) {
    if (ctr->done) return;
    const unsigned d = ctr->d;
    const long long acc = (long long)ctr->accepted;
    if (ctr->fovf || ctr->guard) {
        ctr->fallback = 1;
        ctr->done = 1;
        return;
    }
    if (d < PLB_MAX_ROUNDS) {
        RoundStat& r = stats[d];
        r.receivers = ctr->nR + ctr->nO1_base;
        r.accepted = acc;
        r.uniq = (long long)ctr->uniq;
        r.probed = (long long)ctr->probed;
        r.msgs = (long long)ctr->msgs;
        r.pref = (long long)ctr->prefiltered;
        r.arcs = (long long)ctr->arcs;
        r.staged = (long long)ctr->staged;
        r.tier0 = (long long)ctr->tier[0];
        r.tier1 = (long long)ctr->tier[1];
    }
    if (acc == 0) {
        ctr->done = 1;
        return;
    }
    if (d > PLB_MAX_DIST) {
        ctr->err = PLB_ERR_DIST_OVERFLOW;
        ctr->done = 1;
        return;
    }
    const long long T = ctr->T + acc;
    if (T > ctr->lcap || 4 * T > ctr->hcap) {  // the merge or the probe index would not fit
        ctr->fallback = 1;
        ctr->done = 1;
        return;
    }
    ctr->T = T;
}

// End of a completed round: flip the buffer parity, clear the per-round counters.
__global__ void k_g_finish(RoundCounters* ctr) {
    if (ctr->done) return;
    ctr->cur ^= 1;
    ctr->cursor = ctr->accepted = ctr->arcs = ctr->msgs = ctr->uniq = ctr->staged = ctr->probed = 0;
    ctr->tier[0] = ctr->tier[1] = ctr->tier[2] = 0;
    ctr->bound_sum = ctr->prefiltered = 0;
    ctr->nR = ctr->nO1 = ctr->nO2 = ctr->nBig = ctr->nGiant = 0;
    ctr->nO1_base = ctr->nO2_base = ctr->fovf = 0;
}

// Loop condition of the graph: continue while not done.
__global__ void k_g_cond(const RoundCounters* ctr, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, ctr->done ? 0u : 1u);
}

// ------------------------------------------------------------ finalize
__global__ void k_final_len(const int64_t* loff, const int32_t* inv, int64_t n, int64_t* len) {
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < n; id += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = inv[id];
        len[id] = loff[r + 1] - loff[r];
    }
}

// Rows by original id: packed copy + separate hub / dist arrays.
__global__ void k_finalize(const int64_t* loff, const uint32_t* lent, const int32_t* inv, const int64_t* out_off,
                           uint32_t* out_packed, uint32_t* out_hub, uint8_t* out_dist, int64_t n,
                           RoundCounters* ctr) {
    __shared__ int64_t sh_r[2];
    const int64_t total = out_off[n];
    const int64_t ntiles = (total + kTileItems - 1) / kTileItems;
    uint32_t md = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(total, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(out_off, n, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        for (int64_t q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
            const int64_t id = row_of(out_off, r0, r1, q);
            const int32_t r = inv[id];
            const uint32_t e = lent[loff[r] + (q - out_off[id])];
            out_packed[q] = e;
            out_hub[q] = hub_of(e);
            out_dist[q] = (uint8_t)dist_of(e);
            md = max(md, dist_of(e));
        }
    }
    md = max(md, __shfl_xor_sync(kFull, md, 16));
    md = max(md, __shfl_xor_sync(kFull, md, 8));
    md = max(md, __shfl_xor_sync(kFull, md, 4));
    md = max(md, __shfl_xor_sync(kFull, md, 2));
    md = max(md, __shfl_xor_sync(kFull, md, 1));
    if ((threadIdx.x & 31) == 0 && md) atomicMax(&ctr->max_dist, md);
}

}  // namespace plb
