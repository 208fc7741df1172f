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

// Flat over the arcs of the active list: flag v in N(a) if min dL(a) < v.
__global__ void k_mark(const int64_t* roff, const int32_t* rcol, const uint64_t* fse, const uint32_t* fhub,
                       const int32_t* A, const int64_t* aoff, const RoundCounters* ctr, uint8_t* recv, int64_t n) {
    __shared__ int64_t sh_r[2];
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
            const uint32_t minh = fhub[fstart(fse[a])];
            const int32_t v = rcol[roff[a] + (p - aoff[i])];
            if ((uint32_t)v > minh) recv[v] = 1;
        }
    }
}

// Receivers: flagged vertices.  Vertices with |L(v)| > warp_label_limit or
// degree > warp_deg_limit go to the block tier directly.  Also clears the
// flags and the new frontier descriptors.
__global__ void k_collect(uint8_t* recv, const int64_t* roff, const int64_t* loff, int64_t n, uint64_t* fse_new,
                          int32_t* R, int32_t* O1, RoundCounters* ctr, int64_t warp_label_limit,
                          int64_t warp_deg_limit) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        fse_new[v] = 0;
        const bool r = recv[v] != 0;
        bool heavy = false;
        if (r) {
            recv[v] = 0;
            heavy = (loff[v + 1] - loff[v]) > warp_label_limit || (roff[v + 1] - roff[v]) > warp_deg_limit;
        }
        const unsigned am = __activemask();
        const unsigned mw = __ballot_sync(am, r && !heavy);
        const unsigned mh = __ballot_sync(am, r && heavy);
        const int lane = lane_id();
        if (mw) {
            const int leader = __ffs(mw) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&ctr->nR, __popc(mw));
            base = __shfl_sync(am, base, leader);
            if (r && !heavy) R[base + __popc(mw & ((1u << lane) - 1u))] = (int32_t)v;
        }
        if (mh) {
            const int leader = __ffs(mh) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&ctr->nO1, __popc(mh));
            base = __shfl_sync(am, base, leader);
            if (r && heavy) O1[base + __popc(mh & ((1u << lane) - 1u))] = (int32_t)v;
        }
    }
}

__global__ void k_after_collect(RoundCounters* ctr) {
    ctr->nO1_base = ctr->nO1;
    ctr->nA = 0;
}

// Reset before re-running the gather/prune of a round with a bigger buffer.
__global__ void k_rerun_reset(RoundCounters* ctr, uint64_t* fse_new, int64_t n) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        fse_new[v] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->nO1 = ctr->nO1_base;
        ctr->nO2 = 0;
        ctr->cursor = 0;
        ctr->accepted = 0;
        ctr->fovf = 0;
        ctr->arcs = ctr->msgs = ctr->uniq = ctr->staged = ctr->probed = 0;
        ctr->tier[0] = ctr->tier[1] = ctr->tier[2] = 0;
    }
}

// ------------------------------------------------------- gather + prune
// One warp per vertex v:
//  1. stage L(v) into the hub-keyed map M (shared memory);
//  2. gather: for every neighbour a and every h in dL_{d-1}(a) with h < v and
//     h not already a hub of v, insert h into the set S (unique messages);
//  3. check each h in S: accept iff no w in L(h) has M[w] + d(w,h) <= d
//     (the distance check of Alg. 3 with the labels of round d-1);
//  4. sort the accepted hubs and append them to the new frontier.
// A vertex whose unique candidates exceed cand_limit goes to the next tier.
__global__ void __launch_bounds__(256) k_gp_warp(GpParams p) {
    extern __shared__ uint32_t sm[];
    const int lane = lane_id(), wib = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int S_CAP = 1 << p.log_s, M_CAP = 1 << p.log_m, ACC = p.cand_limit;
    volatile int* wsc = reinterpret_cast<volatile int*>(sm) + wib * 4;
    uint32_t* S = sm + 4 * nwarps + wib * (S_CAP + M_CAP + ACC);
    uint32_t* M = S + S_CAP;
    uint32_t* acc = M + M_CAP;
    unsigned long long c_arcs = 0, c_msgs = 0, c_uniq = 0, c_staged = 0, c_probed = 0, c_acc = 0, c_vert = 0;
    const int nlist = *p.list_n;
    for (int i = blockIdx.x * nwarps + wib; i < nlist; i += gridDim.x * nwarps) {
        __syncwarp();
        const int32_t v = p.list[i];
        const int64_t lb = p.loff[v], ll = p.loff[v + 1] - lb;
        for (int s = lane; s < S_CAP; s += 32) S[s] = kEmpty;
        for (int s = lane; s < M_CAP; s += 32) M[s] = kEmpty;
        if (lane == 0) {
            wsc[0] = 0;
            wsc[1] = 0;
            wsc[2] = 0;
        }
        __syncwarp();
        for (int64_t j = lane; j < ll; j += 32) map_insert(M, p.log_m, p.lent[lb + j]);
        c_staged += ll;
        __syncwarp();
        const int64_t nb = p.roff[v], ne = p.roff[v + 1];
        c_arcs += ne - nb;
        bool ovf = false;
        for (int64_t base = nb; base < ne && !ovf; base += 32) {
            const int64_t j = base + lane;
            int cnt = 0;
            int64_t st = 0;
            if (j < ne) {
                const uint64_t f = p.fse[p.rcol[j]];
                st = (int64_t)fstart(f);
                cnt = (int)fcount(f);
            }
            const int incl = warp_incl_scan(cnt, lane);
            const int total = __shfl_sync(kFull, incl, 31);
            const int excl = incl - cnt;
            c_msgs += total;
            for (int ib = 0; ib < total; ib += 32) {
                const int it = ib + lane;
                const int k = warp_owner(excl, it);
                const int64_t stk = __shfl_sync(kFull, st, k);
                const int exk = __shfl_sync(kFull, excl, k);
                if (it < total) {
                    const uint32_t h = p.fhub[stk + (it - exk)];
                    if (h < (uint32_t)v && map_find(M, p.log_m, h) == kEmpty) {
                        if (wsc[0] >= p.cand_limit) {
                            wsc[1] = 1;
                        } else if (set_insert(S, p.log_s, h)) {
                            atomicAdd((int*)&wsc[0], 1);
                        }
                    }
                }
                __syncwarp();
                if (wsc[1]) {
                    ovf = true;
                    break;
                }
            }
        }
        __syncwarp();
        if (ovf || wsc[0] > p.cand_limit) {
            if (lane == 0) {
                const int o = atomicAdd(p.esc_n, 1);
                p.esc[o] = v;
            }
            continue;
        }
        c_vert += 1;
        c_uniq += wsc[0];
        // distance checks
        for (int sb = 0; sb < S_CAP; sb += 32) {
            const uint32_t h = S[sb + lane];
            const bool has = h != kEmpty;
            unsigned mask = __ballot_sync(kFull, has);
            int64_t hb = 0, he = 0;
            if (has) {
                hb = p.loff[h];
                he = p.loff[h + 1];
            }
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const uint32_t hh = __shfl_sync(kFull, h, src);
                const int64_t b = __shfl_sync(kFull, hb, src), e = __shfl_sync(kFull, he, src);
                bool wit = false;
                for (int64_t jb = b; jb < e; jb += 32) {
                    const int64_t jj = jb + lane;
                    bool hit = false;
                    if (jj < e) {
                        const uint32_t x = p.lent[jj];
                        const uint32_t dv = map_find(M, p.log_m, hub_of(x));
                        hit = dv != kEmpty && dv + dist_of(x) <= p.d;
                    }
                    c_probed += (unsigned long long)min((int64_t)32, e - jb);
                    if (__any_sync(kFull, hit)) {
                        wit = true;
                        break;
                    }
                }
                if (!wit && lane == 0) {
                    const int q = wsc[2];
                    acc[q] = hh;
                    wsc[2] = q + 1;
                }
            }
        }
        __syncwarp();
        const int nacc = wsc[2];
        if (nacc > 0) {
            int P = 1;
            while (P < nacc) P <<= 1;
            for (int s = nacc + lane; s < P; s += 32) acc[s] = kEmpty;
            __syncwarp();
            group_bitonic_sort(acc, P, lane, 32, WarpSync());
            unsigned long long start = 0;
            if (lane == 0) start = atomicAdd(&p.ctr->cursor, (unsigned long long)nacc);
            start = __shfl_sync(kFull, start, 0);
            if (start + nacc <= p.fcap) {
                for (int j = lane; j < nacc; j += 32) p.fhub_new[start + j] = acc[j];
                if (lane == 0) p.fse_new[v] = fpack(start, (uint32_t)nacc);
            } else if (lane == 0) {
                p.ctr->fovf = 1;
            }
            c_acc += nacc;
        }
    }
    if (lane == 0) {
        // per-lane counters that every lane accumulated identically: count once
        atomicAdd(&p.ctr->arcs, c_arcs);
        atomicAdd(&p.ctr->msgs, c_msgs);
        atomicAdd(&p.ctr->uniq, c_uniq);
        atomicAdd(&p.ctr->staged, c_staged);
        atomicAdd(&p.ctr->probed, c_probed);
        atomicAdd(&p.ctr->accepted, c_acc);
        atomicAdd(&p.ctr->tier[0], c_vert);
    }
}

// One block per vertex; tables either in shared memory (kGlobal = false) or
// in this block's slice of global scratch sized for the vertex (kGlobal).
template <bool kGlobal>
__device__ void gp_block_vertex(const GpParams& p, int32_t v, uint32_t* tabs, int log_s_max, int log_m_max,
                                int acc_max, int* sh, unsigned long long* cnt) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    const int64_t lb = p.loff[v], ll = p.loff[v + 1] - lb;
    const int64_t nb = p.roff[v], ne = p.roff[v + 1];
    int log_m = ceil_log2_i64(2 * ll + 2 * nthr);
    if (log_m < 5) log_m = 5;
    int log_s = log_s_max, acc_cap = acc_max;
    if (kGlobal) {
        // bound on unique candidates: min(v, sum of frontier sizes of the neighbours)
        if (tid == 0) sh[3] = 0;
        __syncthreads();
        int64_t part = 0;
        for (int64_t j = nb + tid; j < ne; j += nthr) part += fcount(p.fse[p.rcol[j]]);
        part = warp_sum(part);
        if (lane == 0) atomicAdd((unsigned long long*)(sh + 4), (unsigned long long)part);
        __syncthreads();
        int64_t bound = (int64_t)(*(unsigned long long*)(sh + 4));
        if (bound > v) bound = v;
        log_s = ceil_log2_i64(2 * bound + 2 * nthr);
        if (log_s < 5) log_s = 5;
        acc_cap = 1 << ceil_log2_i64(bound + 1);
        __syncthreads();
        if (tid == 0) *(unsigned long long*)(sh + 4) = 0;
    } else if (log_m > log_m_max) {
        if (tid == 0) {
            const int o = atomicAdd(p.esc_n, 1);
            p.esc[o] = v;
        }
        return;
    }
    const int S_CAP = 1 << log_s, M_CAP = 1 << log_m;
    const int limit = kGlobal ? acc_cap : p.cand_limit;
    uint32_t* S = tabs;
    uint32_t* M = S + S_CAP;
    uint32_t* acc = M + M_CAP;
    for (int s = tid; s < S_CAP; s += nthr) S[s] = kEmpty;
    for (int s = tid; s < M_CAP; s += nthr) M[s] = kEmpty;
    if (tid == 0) {
        sh[0] = 0;  // unique count
        sh[1] = 0;  // overflow
        sh[2] = 0;  // accepted count
    }
    __syncthreads();
    for (int64_t j = tid; j < ll; j += nthr) map_insert(M, log_m, p.lent[lb + j]);
    __syncthreads();
    volatile int* vsh = sh;
    // gather: warp w handles neighbour chunks w, w + nw, ...
    bool stop = false;
    for (int64_t base = nb + 32 * wid; base < ne && !stop; base += 32 * nw) {
        const int64_t j = base + lane;
        int c = 0;
        int64_t st = 0;
        if (j < ne) {
            const uint64_t f = p.fse[p.rcol[j]];
            st = (int64_t)fstart(f);
            c = (int)fcount(f);
        }
        const int incl = warp_incl_scan(c, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - c;
        if (lane == 0) cnt[1] += total;
        for (int ib = 0; ib < total; ib += 32) {
            const int it = ib + lane;
            const int k = warp_owner(excl, it);
            const int64_t stk = __shfl_sync(kFull, st, k);
            const int exk = __shfl_sync(kFull, excl, k);
            if (it < total) {
                const uint32_t h = p.fhub[stk + (it - exk)];
                if (h < (uint32_t)v && map_find(M, log_m, h) == kEmpty) {
                    if (vsh[0] >= limit) {
                        vsh[1] = 1;
                    } else if (set_insert(S, log_s, h)) {
                        atomicAdd(&sh[0], 1);
                    }
                }
            }
            if (__any_sync(kFull, vsh[1] != 0)) {
                stop = true;
                break;
            }
        }
    }
    __syncthreads();
    const int nS = vsh[0];
    if (vsh[1] || nS > limit) {
        __syncthreads();
        if (tid == 0) {
            const int o = atomicAdd(p.esc_n, 1);
            p.esc[o] = v;
        }
        return;
    }
    if (tid == 0) {
        cnt[0] += ne - nb;
        cnt[2] += nS;
        cnt[3] += ll;
        cnt[6] += 1;
    }
    // distance checks: warp w takes slot chunks w, w + nw, ...
    for (int sb = 32 * wid; sb < S_CAP; sb += 32 * nw) {
        const uint32_t h = S[sb + lane];
        const bool has = h != kEmpty;
        unsigned mask = __ballot_sync(kFull, has);
        int64_t hb = 0, he = 0;
        if (has) {
            hb = p.loff[h];
            he = p.loff[h + 1];
        }
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const uint32_t hh = __shfl_sync(kFull, h, src);
            const int64_t b = __shfl_sync(kFull, hb, src), e = __shfl_sync(kFull, he, src);
            bool wit = false;
            for (int64_t jb = b; jb < e; jb += 32) {
                const int64_t jj = jb + lane;
                bool hit = false;
                if (jj < e) {
                    const uint32_t x = p.lent[jj];
                    const uint32_t dv = map_find(M, log_m, hub_of(x));
                    hit = dv != kEmpty && dv + dist_of(x) <= p.d;
                }
                if (lane == 0) cnt[4] += (unsigned long long)min((int64_t)32, e - jb);
                if (__any_sync(kFull, hit)) {
                    wit = true;
                    break;
                }
            }
            if (!wit && lane == 0) {
                const int q = atomicAdd(&sh[2], 1);
                acc[q] = hh;
            }
        }
    }
    __syncthreads();
    const int nacc = vsh[2];
    if (nacc > 0) {
        int P = 1;
        while (P < nacc) P <<= 1;
        for (int s = nacc + tid; s < P; s += nthr) acc[s] = kEmpty;
        __syncthreads();
        group_bitonic_sort(acc, P, tid, nthr, BlockSync());
        if (tid == 0) {
            const unsigned long long start = atomicAdd(&p.ctr->cursor, (unsigned long long)nacc);
            *(unsigned long long*)(sh + 6) = start;
        }
        __syncthreads();
        const unsigned long long start = *(volatile unsigned long long*)(sh + 6);
        if (start + nacc <= p.fcap) {
            for (int j = tid; j < nacc; j += nthr) p.fhub_new[start + j] = acc[j];
            if (tid == 0) p.fse_new[v] = fpack(start, (uint32_t)nacc);
        } else if (tid == 0) {
            p.ctr->fovf = 1;
        }
        if (tid == 0) cnt[5] += nacc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_gp_block(GpParams p) {
    extern __shared__ uint32_t sm[];
    int* sh = reinterpret_cast<int*>(sm);            // 16 ints of scalars
    uint32_t* tabs = sm + 16;
    unsigned long long cnt[7] = {0, 0, 0, 0, 0, 0, 0};
    const int n1 = *p.list_n;
    for (int i = blockIdx.x; i < n1; i += gridDim.x) {
        gp_block_vertex<false>(p, p.list[i], tabs, p.log_s, p.log_m, p.cand_limit, sh, cnt);
        __syncthreads();
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&p.ctr->msgs, cnt[1]);
        atomicAdd(&p.ctr->probed, cnt[4]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&p.ctr->arcs, cnt[0]);
        atomicAdd(&p.ctr->uniq, cnt[2]);
        atomicAdd(&p.ctr->staged, cnt[3]);
        atomicAdd(&p.ctr->accepted, cnt[5]);
        atomicAdd(&p.ctr->tier[1], cnt[6]);
    }
}

__global__ void __launch_bounds__(1024) k_gp_global(GpParams p) {
    __shared__ __align__(8) int sh[16];
    unsigned long long cnt[7] = {0, 0, 0, 0, 0, 0, 0};
    const int n2 = *p.list_n;
    uint32_t* tabs = p.gscratch + (int64_t)blockIdx.x * p.gscratch_words;
    if (threadIdx.x == 0) *(unsigned long long*)(sh + 4) = 0;
    __syncthreads();
    for (int i = blockIdx.x; i < n2; i += gridDim.x) {
        gp_block_vertex<true>(p, p.list[i], tabs, 0, 0, 0, sh, cnt);
        __syncthreads();
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&p.ctr->msgs, cnt[1]);
        atomicAdd(&p.ctr->probed, cnt[4]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&p.ctr->arcs, cnt[0]);
        atomicAdd(&p.ctr->uniq, cnt[2]);
        atomicAdd(&p.ctr->staged, cnt[3]);
        atomicAdd(&p.ctr->accepted, cnt[5]);
        atomicAdd(&p.ctr->tier[2], cnt[6]);
    }
}

// ------------------------------------------------------------ merge
// next active list + per-vertex new row lengths
__global__ void k_next_active(const int64_t* loff, const uint64_t* fse_new, int64_t n, int64_t* newlen, int32_t* A,
                              RoundCounters* ctr) {
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

// Old entries move to their place in the merged row: flat over old entries.
__global__ void k_merge_old(const int64_t* loff, const uint32_t* lent, const int64_t* loff_new, uint32_t* lent_new,
                            const uint64_t* fse_new, const uint32_t* fhub_new, int64_t n) {
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
                            const RoundCounters* ctr, uint32_t d) {
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
        }
    }
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
