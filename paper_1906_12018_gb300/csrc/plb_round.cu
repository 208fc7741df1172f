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

// Per arc (u -> c): 0 <= c < n, c != u, rows strictly ascending, and (when
// symmetric) the reverse arc (c -> u) exists (binary search in row c).
__global__ void k_check_cols(const int64_t* row_ptr, const int32_t* col, int64_t n, int64_t nnz, int symmetric,
                             int* err) {
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
            if (!bad && symmetric) {
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

// ------------------------------------------------------------ transpose
// In-degrees of the rank-space arcs (indeg zeroed by the caller).
__global__ void k_in_degree(const int32_t* rcol, int64_t nnz, int64_t* indeg) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long*)&indeg[rcol[p]], 1ull);
}

// rcol_t: the transpose of (roff, rcol) at row offsets roff_t; fill[] counts
// the entries placed per row (zeroed by the caller; rows come out unsorted).
__global__ void k_transpose(const int64_t* roff, const int32_t* rcol, int64_t n, int64_t nnz, const int64_t* roff_t,
                            unsigned long long* fill, int32_t* rcol_t) {
    __shared__ int64_t sh_r[2];
    const int64_t ntiles = (nnz + kTileItems - 1) / kTileItems;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(nnz, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(roff, n, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int64_t u = row_of(roff, r0, r1, p);
            const int32_t w = rcol[p];
            rcol_t[roff_t[w] + (int64_t)atomicAdd(&fill[w], 1ull)] = (int32_t)u;
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
// rbound[v] (it sizes the warp tier's tables) and, when obound is given, in
// obound[v] for every v (0 for non-receivers: its scan places each row of the
// new frontier).  Also clears recv and the new frontier descriptors, and sums
// the bounds.
__global__ void k_collect(unsigned long long* recv, const int64_t* roff, const int64_t* loff, int64_t n,
                          uint64_t* fse_new, int32_t* R, int32_t* O1, uint32_t* rbound, int64_t* obound,
                          RoundCounters* ctr, TierLimits lim) {
    if (ctr->done) return;
    unsigned long long bsum = 0;
    const int lane = lane_id();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        fse_new[v] = 0;
        const unsigned long long c = recv[v];
        int tier = -1;
        if (obound) obound[v] = c < (unsigned long long)v ? (int64_t)c : v;
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

// Round 1 (Alg. 3 with d = 1) of the hubs [s, e) (all hubs, or one batch of
// Alg. 4).  The candidates of v are its neighbours a in [s, e) with a < v
// (each sends its label (a, 0)), they are distinct, and none is pruned: a
// witness w of (a, 1) at v would need d(w, v) + d(w, a) <= 1, so w = v or
// w = a, but (v, .) is not a hub of a (v > a) and (a, .) not yet one of v.
// So dL_1(v) = N(v) n [s, min(e, v)): it is appended (unsorted; the merge
// step sorts the rows), the other frontier descriptors are cleared and the
// active list restarts.  Counted like the general round:
// one message, one unique candidate and one accepted label per such neighbour.
// Both passes run flat over tiles of arcs (a hub's row is spread over many
// warps instead of one), each arc's row found by binary search in the tile's
// row range.
// Count pass: cnt[v] = |N(v) n [s, min(e, v))| (cnt zero on entry; one
// atomic per row and warp).
__global__ void k_round1_count(const int64_t* roff, const int32_t* rcol, int64_t n, int64_t nnz, int32_t s,
                               int32_t e, unsigned long long* cnt, const RoundCounters* ctr) {
    __shared__ int64_t sh_r[2];
    if (ctr->done) return;
    const int lane = lane_id();
    const int64_t ntiles = (nnz + kTileItems - 1) / kTileItems;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(nnz, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(roff, n, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        for (int64_t q = p0; q < p1; q += blockDim.x) {  // uniform trip count: whole warps below
            const int64_t p = q + threadIdx.x;
            const bool ok = p < p1;
            int64_t v = -1;
            int c = 0;
            if (ok) {
                v = row_of(roff, r0, r1, p);
                const int32_t a = rcol[p];
                c = (a >= s && a < e && (int64_t)a < v) ? 1 : 0;
            }
            int first, last;
            const int sum = run_sum(v, c, lane, &first, &last);
            if (ok && lane == last && sum > 0) atomicAdd(cnt + v, (unsigned long long)sum);
        }
    }
}

// Write pass: row v of the new frontier at start[v] (the exclusive scan of
// the counts: no shared cursor), start[n] entries in all; within a row the
// entries are placed by the per-row cursor cur[v] (zero on entry; one atomic
// per row and warp).  Then, per vertex, the frontier descriptor and the
// counters.
__global__ void k_round1(const int64_t* roff, const int32_t* rcol, int64_t n, int64_t nnz, int32_t s, int32_t e,
                         const int64_t* start, uint32_t* cur, uint64_t* fse_new, uint32_t* fhub_new,
                         unsigned long long fcap, RoundCounters* ctr) {
    __shared__ int64_t sh_r[2];
    if (ctr->done) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->nA_saved = ctr->nA;
        ctr->nA = 0;
        if ((unsigned long long)start[n] > fcap) ctr->fovf = 1;  // cannot happen: the buffer holds every arc
        else ctr->cursor = (unsigned long long)start[n];
    }
    if ((unsigned long long)start[n] > fcap) return;
    const int lane = lane_id();
    const int64_t ntiles = (nnz + kTileItems - 1) / kTileItems;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(nnz, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(roff, n, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        for (int64_t q = p0; q < p1; q += blockDim.x) {
            const int64_t p = q + threadIdx.x;
            const bool ok = p < p1;
            int64_t v = -1;
            int32_t a = 0;
            bool up = false;
            if (ok) {
                v = row_of(roff, r0, r1, p);
                a = rcol[p];
                up = a >= s && a < e && (int64_t)a < v;
            }
            int first, last;
            const int cnt = run_sum(v, up ? 1 : 0, lane, &first, &last);
            const unsigned upm = __ballot_sync(kFull, up);
            unsigned base = 0;
            if (ok && lane == first && cnt > 0) base = atomicAdd(cur + v, (unsigned)cnt);
            base = __shfl_sync(kFull, base, first);
            if (up) {
                const unsigned below = upm & ((1u << lane) - 1u) & ~((1u << first) - 1u);
                fhub_new[start[v] + base + __popc(below)] = (uint32_t)a;
            }
        }
    }
    unsigned long long c_acc = 0, c_arcs = 0, c_recv = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t st = start[v];
        const int64_t c = start[v + 1] - st;
        fse_new[v] = c ? fpack((uint64_t)st, (uint32_t)c) : 0ull;
        if (c) {
            c_acc += (unsigned long long)c;
            c_arcs += (unsigned long long)(roff[v + 1] - roff[v]);
            c_recv += 1;
        }
    }
    c_acc = warp_sum(c_acc);
    c_arcs = warp_sum(c_arcs);
    c_recv = warp_sum(c_recv);
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
        ctr->nU = 0;
        ctr->arcs = ctr->msgs = ctr->uniq = ctr->staged = ctr->probed = ctr->chk_lv = ctr->chk_lh = 0;
        ctr->tier[0] = ctr->tier[1] = ctr->tier[2] = 0;
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

// Build the table of the sorted row lent[lb, lb + ll) at htab[hb, hb + 2^lg):
// in the warp's shared-memory buffer when it has up to `slots` slots (then
// written out whole, empty slots included), else cleared and filled in place.
__device__ __forceinline__ void build_table(const uint32_t* lent, int64_t lb, int64_t ll, uint32_t* htab,
                                            int64_t hb, int lg, uint32_t* buf, int slots, int lane) {
    const int P = 1 << lg;
    uint32_t* tab = P <= slots ? buf : htab + hb;
    for (int sl = lane; sl < P; sl += 32) tab[sl] = kEmpty;
    __syncwarp();
    for (int64_t j = lane; j < ll; j += 32) map_insert(tab, lg, lent[lb + j]);
    __syncwarp();
    if (P <= slots) {
        for (int sl = lane; sl < P; sl += 32) htab[hb + sl] = buf[sl];
        __syncwarp();
    }
}

// Full rebuild, one warp per 32 rows: row x's table at hoff[x] (sizes from
// k_index_size and a scan); hdesc[x] = hoff[x] << 8 | log2 size, or 0.
__global__ void __launch_bounds__(kIndexWarps * 32) k_index_build(const int64_t* loff, const uint32_t* lent,
                                                                  const int64_t* hoff, uint32_t* htab,
                                                                  uint64_t* hdesc, int64_t n, int slots,
                                                                  const RoundCounters* ctr) {
    extern __shared__ uint32_t ibuf[];
    if (ctr->done) return;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    uint32_t* buf = ibuf + w * slots;
    const int64_t nwarps = (int64_t)gridDim.x * kIndexWarps;
    for (int64_t base = ((int64_t)blockIdx.x * kIndexWarps + w) * 32; base < n; base += nwarps * 32) {
        const int64_t x = base + lane;
        int64_t hb = 0, P = 0;
        if (x < n) {
            hb = hoff[x];
            P = hoff[x + 1] - hb;
            hdesc[x] = P > 0 ? ((uint64_t)hb << 8) | (uint64_t)(__ffsll((unsigned long long)P) - 1) : 0ull;
        }
        unsigned m = __ballot_sync(kFull, P > 0);
        while (m) {
            const int k = __ffs(m) - 1;
            m &= m - 1;
            const int64_t xk = base + k;
            const int64_t hbk = __shfl_sync(kFull, hb, k);
            const int Pk = (int)__shfl_sync(kFull, P, k);
            const int64_t lb = loff[xk], ll = loff[xk + 1] - lb;
            build_table(lent, lb, ll, htab, hbk, __ffs(Pk) - 1, buf, slots, lane);
        }
    }
}

// After a full rebuild: the next free slot of the table pool.
__global__ void k_index_total(const int64_t* hoff, int64_t n, RoundCounters* ctr) {
    if (ctr->done) return;
    ctr->hnext = hoff[n];
    ctr->hovf = 0;
}

// Incremental update after a merge, one warp per row that changed (the new
// active list A): a row whose table still has room (size >= 2 |L(x)|) gets
// this round's new entries (hubs of the new frontier row, distance d) inserted;
// a row that outgrew its table, or reached kIndexMinLen entries, gets a new
// table from the pool (the old one is left unused).  A table that does not fit
// the pool sets hovf: the caller rebuilds the whole index before its next use.
__global__ void __launch_bounds__(kIndexWarps * 32) k_index_update(const int64_t* loff, const uint32_t* lent,
                                                                   const uint64_t* fse_new, const uint32_t* fhub_new,
                                                                   const int32_t* A, uint32_t* htab, uint64_t* hdesc,
                                                                   long long hcap, int slots, RoundCounters* ctr) {
    extern __shared__ uint32_t ibuf[];
    if (ctr->done) return;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    uint32_t* buf = ibuf + w * slots;
    const uint32_t d = ctr->d;
    const int nA = ctr->nA;
    const int nwarps = gridDim.x * kIndexWarps;
    for (int i = blockIdx.x * kIndexWarps + w; i < nA; i += nwarps) {
        const int32_t x = A[i];
        const int64_t lb = loff[x], ll = loff[x + 1] - lb;
        if (ll < kIndexMinLen) continue;
        const int lgn = ceil_log2_i64(2 * ll);
        const uint64_t hd = hdesc[x];
        if (hd != 0 && (int)(hd & 0xFFu) >= lgn) {
            const uint64_t f = fse_new[x];
            const uint32_t* row = fhub_new + fstart(f);
            const int c = (int)fcount(f), lg = (int)(hd & 0xFFu);
            uint32_t* tab = htab + (hd >> 8);
            for (int j = lane; j < c; j += 32) map_insert(tab, lg, pack(row[j], d));
            continue;
        }
        long long hb = 0;
        if (lane == 0) hb = (long long)atomicAdd((unsigned long long*)&ctr->hnext, 1ull << lgn);
        hb = __shfl_sync(kFull, hb, 0);
        if (hb + ((long long)1 << lgn) > hcap) {
            if (lane == 0) ctr->hovf = 1;
            continue;
        }
        build_table(lent, lb, ll, htab, hb, lgn, buf, slots, lane);
        if (lane == 0) hdesc[x] = ((uint64_t)hb << 8) | (uint64_t)lgn;
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

// The rows taken: every new row (A, ctr->nA) when U is null or, with
// r1_all, in round 1 (whose rows k_round1 writes unsorted); else the rows the
// block tier listed in U (ctr->nU).
__global__ void __launch_bounds__(kSortWarps * 32) k_sort_rows_warp(const uint64_t* fse_new, uint32_t* fhub_new,
                                                                   const int32_t* A, const int32_t* U, int r1_all,
                                                                   RoundCounters* ctr, int32_t* big,
                                                                   int32_t* giant) {
    __shared__ uint32_t buf[kSortWarps][kWarpSortMax];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    if (ctr->done) return;
    const bool all = U == nullptr || (r1_all && ctr->d == 1);
    const int nA = all ? ctr->nA : ctr->nU;
    if (!all) A = U;
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

// Rows of kWarpSortMax < c <= kBlockSortSmem entries (the list k_sort_rows_warp
// makes): one block of kRadixThreads per row, an LSD radix sort in shared
// memory on the three 8-bit digits of a hub rank (below 2^24).  Each pass is
// stable: warp w owns the w-th
// contiguous chunk of the row and reads it 32 entries at a time in order;
// lanes with equal digits find one another with __match_any_sync.  A count
// pass fills a (digit, warp) histogram, its exclusive scan in digit-major
// order gives every warp its first slot per digit, and a scatter pass writes
// each entry at that slot plus its rank among the earlier equal digits.
constexpr int kRadixThreads = 1024;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixBins = 256;
static_assert(kRadixBins * kRadixWarps % kRadixThreads == 0, "histogram scan: whole entries per thread");
static_assert(kSortRadixSmemBytes == (2 * kBlockSortSmem + (kRadixBins + 1) * kRadixWarps) * (int)sizeof(uint32_t),
              "launch size of k_sort_rows_radix");

__global__ void __launch_bounds__(kRadixThreads) k_sort_rows_radix(const uint64_t* fse_new, uint32_t* fhub_new,
                                                                  const int32_t* big, const int* nbig,
                                                                  const RoundCounters* ctr) {
    extern __shared__ uint32_t sbuf[];
    uint32_t* buf0 = sbuf;                                                     // kBlockSortSmem
    uint32_t* buf1 = sbuf + kBlockSortSmem;                                    // kBlockSortSmem
    // (digit, warp) counts, warp-major with a padded row: the digits a warp's
    // lanes touch at once fall in different banks
    int* hist = reinterpret_cast<int*>(sbuf + 2 * kBlockSortSmem);             // [kRadixWarps][kRadixBins + 1]
    auto hidx = [](uint32_t dg, int ww) { return ww * (kRadixBins + 1) + (int)dg; };
    __shared__ int wtot[kRadixWarps];
    constexpr int kPer = kRadixBins * kRadixWarps / kRadixThreads;            // histogram entries per thread
    if (ctr->done) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nBig = *nbig;
    for (int i = blockIdx.x; i < nBig; i += gridDim.x) {
        const uint64_t f = fse_new[big[i]];
        const int c = min((int)fcount(f), kBlockSortSmem);  // (the list holds rows of at most kBlockSortSmem)
        uint32_t* row = fhub_new + fstart(f);
        constexpr int passes = 3;  // hub ranks below 2^24
        for (int j = threadIdx.x; j < c; j += kRadixThreads) buf0[j] = row[j];
        const int chunk = (c + kRadixWarps - 1) / kRadixWarps;
        const int wb = min(c, w * chunk), we = min(c, wb + chunk);
        uint32_t* src = buf0;
        uint32_t* dst = buf1;
        for (int pass = 0; pass < passes; ++pass) {
            const int shift = 8 * pass;
            for (int j = threadIdx.x; j < (kRadixBins + 1) * kRadixWarps; j += kRadixThreads) hist[j] = 0;
            __syncthreads();  // (and the row is loaded)
            for (int b0 = wb; b0 < we; b0 += 32) {
                const int j = b0 + lane;
                const bool in = j < we;
                const uint32_t dg = in ? (src[j] >> shift) & (kRadixBins - 1) : (uint32_t)kRadixBins;
                const unsigned peers = __match_any_sync(kFull, dg);
                if (in && (peers & lt) == 0u) hist[hidx(dg, w)] += __popc(peers);
                __syncwarp();
            }
            __syncthreads();
            {  // exclusive scan of the histogram in place, in digit-major order
                int x[kPer], sum = 0;
#pragma unroll
                for (int k = 0; k < kPer; ++k) {
                    const int pos = threadIdx.x * kPer + k;
                    x[k] = hist[hidx(pos / kRadixWarps, pos % kRadixWarps)];
                    sum += x[k];
                }
                const int incl = warp_incl_scan(sum, lane);
                if (lane == 31) wtot[w] = incl;
                __syncthreads();
                if (w == 0) {
                    const int t = wtot[lane];
                    const int ti = warp_incl_scan(t, lane);
                    __syncwarp();
                    wtot[lane] = ti - t;
                }
                __syncthreads();
                int run = wtot[w] + incl - sum;
#pragma unroll
                for (int k = 0; k < kPer; ++k) {
                    const int pos = threadIdx.x * kPer + k;
                    hist[hidx(pos / kRadixWarps, pos % kRadixWarps)] = run;
                    run += x[k];
                }
            }
            __syncthreads();
            for (int b0 = wb; b0 < we; b0 += 32) {
                const int j = b0 + lane;
                const bool in = j < we;
                const uint32_t x = in ? src[j] : 0u;
                const uint32_t dg = in ? (x >> shift) & (kRadixBins - 1) : (uint32_t)kRadixBins;
                const unsigned peers = __match_any_sync(kFull, dg);
                const int leader = __ffs(peers) - 1;
                int base = 0;
                if (in && lane == leader) base = hist[hidx(dg, w)];
                base = __shfl_sync(kFull, base, leader);
                if (in) dst[base + __popc(peers & lt)] = x;
                __syncwarp();
                if (in && lane == leader) hist[hidx(dg, w)] = base + __popc(peers);
                __syncwarp();
            }
            __syncthreads();  // every warp is done with this pass's histogram and output
            uint32_t* t = src;
            src = dst;
            dst = t;
        }
        for (int j = threadIdx.x; j < c; j += kRadixThreads) row[j] = src[j];
        __syncthreads();
    }
}

// Old entries move to their place in the merged row: flat over old entries.
// A tile of entries that spans at most kMergeRows rows stages those rows'
// old and new offsets and new-frontier descriptors in shared memory (each
// entry's row is a binary search there); a tile over more rows reads them
// from global memory.
constexpr int kMergeRows = 512;

__global__ void k_merge_old(const int64_t* loff, const uint32_t* lent, const int64_t* loff_new, uint32_t* lent_new,
                            const uint64_t* fse_new, const uint32_t* fhub_new, int64_t n, const RoundCounters* ctr) {
    __shared__ int64_t sh_r[2];
    __shared__ int64_t s_off[kMergeRows + 1];
    __shared__ int64_t s_noff[kMergeRows];
    __shared__ uint64_t s_f[kMergeRows];
    if (ctr->done) return;
    const int64_t total = loff[n];
    const int64_t ntiles = (total + kTileItems - 1) / kTileItems;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(total, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(loff, n, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        const int64_t rows = r1 - r0 + 1;
        const int nr = rows <= kMergeRows ? (int)rows : kMergeRows + 1;
        const bool staged = nr <= kMergeRows;
        if (staged) {
            for (int i = threadIdx.x; i <= nr; i += blockDim.x) s_off[i] = loff[r0 + i];
            for (int i = threadIdx.x; i < nr; i += blockDim.x) {
                s_noff[i] = loff_new[r0 + i];
                s_f[i] = fse_new[r0 + i];
            }
        }
        __syncthreads();
        for (int64_t q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
            int64_t ob, nb;
            uint64_t f;
            if (staged) {
                int lo = 0, hi = nr - 1;  // last row of the tile whose offset is <= q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= q) lo = mid; else hi = mid - 1;
                }
                ob = s_off[lo];
                nb = s_noff[lo];
                f = s_f[lo];
            } else {
                const int64_t v = row_of(loff, r0, r1, q);
                ob = loff[v];
                nb = loff_new[v];
                f = fse_new[v];
            }
            const uint32_t e = lent[q];
            int64_t pos = nb + (q - ob);
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
        // an old row of at most 32 entries sits in the lanes' registers: the
        // old hubs below h are counted with shuffles instead of a binary
        // search in global memory (c and ol are the same in every lane)
        const bool reg = ol <= 32;
        const uint32_t oe = reg && lane < ol ? lent[ob + lane] : 0xFFFFFFFFu;
        for (uint32_t j0 = 0; j0 < c; j0 += 32) {
            const uint32_t j = j0 + lane;
            const uint32_t h = j < c ? fr[j] : 0u;
            int64_t below;
            if (reg) {
                int cnt = 0;
                for (int k = 0; k < (int)ol; ++k) cnt += __shfl_sync(kFull, oe, k) < pack(h, 0) ? 1 : 0;
                below = cnt;
            } else {
                below = j < c ? lower_bound_u32(lent + ob, ol, pack(h, 0)) : 0;
            }
            if (j >= c) continue;
            const int64_t pos = loff_new[v] + j + below;
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
        r.chk_lv = (long long)ctr->chk_lv;
        r.chk_lh = (long long)ctr->chk_lh;
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
    if (T > ctr->lcap) {  // the merge would not fit
        ctr->fallback = 1;
        ctr->done = 1;
        return;
    }
    ctr->T = T;
}

// End of a completed round: flip the buffer parity, clear the per-round counters.
__global__ void k_g_finish(RoundCounters* ctr) {
    if (ctr->done) return;
    if (ctr->hovf) {  // the round is complete; the host rebuilds the probe index and resumes
        ctr->fallback = kStopIndex;
        ctr->done = 1;
    }
    ctr->cur ^= 1;
    ctr->cursor = ctr->accepted = ctr->arcs = ctr->msgs = ctr->uniq = ctr->staged = ctr->probed = ctr->chk_lv = ctr->chk_lh = 0;
    ctr->tier[0] = ctr->tier[1] = ctr->tier[2] = 0;
    ctr->bound_sum = ctr->prefiltered = 0;
    ctr->nR = ctr->nO1 = ctr->nO2 = ctr->nBig = ctr->nGiant = ctr->nU = 0;
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
    __shared__ int64_t s_off[kMergeRows + 1];  // out_off of the tile's rows (as in k_merge_old)
    __shared__ int64_t s_src[kMergeRows];      // start of each row in rank space
    const int64_t total = out_off[n];
    const int64_t ntiles = (total + kTileItems - 1) / kTileItems;
    uint32_t md = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kTileItems, p1 = min(total, p0 + kTileItems);
        __syncthreads();
        if (threadIdx.x == 0) tile_rows(out_off, n, p0, p1, &sh_r[0], &sh_r[1]);
        __syncthreads();
        const int64_t r0 = sh_r[0], r1 = sh_r[1];
        const int64_t rows = r1 - r0 + 1;
        const int nr = rows <= kMergeRows ? (int)rows : kMergeRows + 1;
        const bool staged = nr <= kMergeRows;
        if (staged) {
            for (int i = threadIdx.x; i <= nr; i += blockDim.x) s_off[i] = out_off[r0 + i];
            for (int i = threadIdx.x; i < nr; i += blockDim.x) s_src[i] = loff[inv[r0 + i]];
        }
        __syncthreads();
        for (int64_t q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
            int64_t src;
            if (staged) {
                int lo = 0, hi = nr - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= q) lo = mid; else hi = mid - 1;
                }
                src = s_src[lo] + (q - s_off[lo]);
            } else {
                const int64_t id = row_of(out_off, r0, r1, q);
                src = loff[inv[id]] + (q - out_off[id]);
            }
            const uint32_t e = lent[src];
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
