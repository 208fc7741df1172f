// Weighted graphs (Sec. 5.1): the canonical labels of Def. 2 over weighted
// shortest paths, (h, d(h, v)) in L(v) iff h outranks every vertex of every
// shortest h-v path, for positive integer arc weights (uint8, equal in both
// directions).
//
// Rounds follow the distance, not the hop count: round d accepts exactly the
// labels at distance d.  A candidate (h, d) at v comes from a neighbour a
// whose round-(d - w) frontier holds h, w = w(a, v); with weights >= 1 every
// label at distance below d is final when round d runs, so the snapshot check
// of Alg. 3 (prune iff some w in L(h) and L(v) has d(h, w) + d(w, v) <= d, with
// both labels read as of round d - 1) is exact, as in the unweighted proof:
// the highest-ranked vertex of all shortest h-v paths is a hub of both h and
// v at distances in [1, d - 1], and a candidate above d(h, v) is pruned by
// (h, d(h, v)) itself or by that vertex.  Accepted rows are therefore the
// canonical ones and no recheck pass is needed (the paper's weighted form
// propagates d + w by hops and rechecks at the end of each batch).
//
// The frontiers of the last maxw rounds stay live: descriptors in a ring of
// S = maxw + 1 slots (slot r mod S holds round r), rows in one append-only
// store in round order (a row start is an absolute offset); slot k's
// descriptors sit at k << lgn, lgn = ceil(log2 n).  Per round a pull pass
// writes each arc's virtual sender, (r mod S) << lgn | a for r = d - w >= 0
// (else the always-empty descriptor S << lgn), and counts the messages of
// every receiver; the gather/prune kernels of the unweighted build then read
// the frontier rows through the virtual senders (GpParams::sender_bits = lgn
// gives them the sending vertex back).  Host-driven rounds, one batch.
#include <algorithm>
#include <cstring>
#include <vector>

#include "plb_host.cuh"

namespace plb {

namespace {

constexpr int kWFlatThreads = 256;

__device__ __forceinline__ int wlane() { return threadIdx.x & 31; }

// mm[0] = min weight, mm[1] = max weight over the nnz arcs.
__global__ void k_weight_range(const uint8_t* wt, int64_t nnz, int* mm) {
    int lo = 255, hi = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x) {
        const int w = wt[j];
        lo = min(lo, w);
        hi = max(hi, w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(kFull, lo, o));
        hi = max(hi, __shfl_xor_sync(kFull, hi, o));
    }
    if (wlane() == 0) {
        atomicMin(mm, lo);
        atomicMax(mm + 1, hi);
    }
}

// Flat kernels over the arcs: tiles of kWTile consecutive arcs, the tile's
// first and last row found once, each arc's row by binary search between
// them (rows of any length are spread evenly over the threads).
constexpr int kWTile = 2048;

__device__ __forceinline__ void tile_bounds(const int64_t* off, int64_t n, int64_t p0, int64_t p1, int64_t* sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        sh[0] = row_of(off, 0, n - 1, p0);
        sh[1] = row_of(off, 0, n - 1, p1 - 1);
    }
    __syncthreads();
}

// Per arc (u -> c) of a validated symmetric CSR: the reverse arc (c -> u),
// found by binary search in row c, has the same weight.
__global__ void k_check_weights(const int64_t* row_ptr, const int32_t* col, const uint8_t* wt, int64_t n,
                                int64_t nnz, int* err) {
    __shared__ int64_t sh[2];
    const int64_t ntiles = (nnz + kWTile - 1) / kWTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kWTile, p1 = min(nnz, p0 + kWTile);
        tile_bounds(row_ptr, n, p0, p1, sh);
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int64_t u = row_of(row_ptr, sh[0], sh[1], p);
            const int32_t c = col[p];
            int64_t lo = row_ptr[c], hi = row_ptr[c + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if ((int64_t)col[mid] < u) lo = mid + 1; else hi = mid;
            }
            if (lo >= row_ptr[c + 1] || (int64_t)col[lo] != u || wt[lo] != wt[p]) atomicOr(err, 1);
        }
    }
}

// Rank-space weights: rwt[p] for arc p of row r = weight of the same arc of
// order[r] (k_relabel keeps the row order).
__global__ void k_relabel_weights(const int64_t* row_ptr, const uint8_t* wt, const int32_t* order,
                                  const int64_t* roff, uint8_t* rwt, int64_t n, int64_t nnz) {
    __shared__ int64_t sh[2];
    const int64_t ntiles = (nnz + kWTile - 1) / kWTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kWTile, p1 = min(nnz, p0 + kWTile);
        tile_bounds(roff, n, p0, p1, sh);
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int64_t r = row_of(roff, sh[0], sh[1], p);
            rwt[p] = wt[row_ptr[order[r]] + (p - roff[r])];
        }
    }
}

// Round d, flat over the receivers' arcs: arc (v, a, w) gets its virtual
// sender ((d - w) mod S) << lgn | a, the descriptor of a's frontier of round
// d - w (or the empty one when d < w),
// and recv[v] += |dL_{d-w}(a)| when that row's smallest hub outranks v (an
// upper bound on v's messages, as in k_mark).  Lanes of a warp that share a
// row add their counts first (one atomic per row and warp; counts are below
// 2^24, a warp's sum below 2^29).  recv is zero on entry (k_collect clears
// what it reads).
__global__ void k_w_pull(const int64_t* roff, const int32_t* rcol, const uint8_t* rwt, int64_t n, int64_t nnz,
                         uint32_t d, int S, int lgn, const uint64_t* fse_ring, const uint32_t* store, int32_t* vcol,
                         unsigned long long* recv) {
    __shared__ int64_t sh[2];
    const int32_t empty = (int32_t)((int64_t)S << lgn);
    const int64_t ntiles = (nnz + kWTile - 1) / kWTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kWTile, p1 = min(nnz, p0 + kWTile);
        tile_bounds(roff, n, p0, p1, sh);
        for (int64_t q = p0; q < p1; q += blockDim.x) {  // uniform trip count: whole warps below
            const int64_t p = q + threadIdx.x;
            const bool ok = p < p1;
            int64_t v = -1;
            unsigned c = 0;
            if (ok) {
                v = row_of(roff, sh[0], sh[1], p);
                const int32_t a = rcol[p];
                const int r = (int)d - (int)rwt[p];
                const int32_t idx = r >= 0 ? (int32_t)(((int64_t)(r % S) << lgn) | a) : empty;
                vcol[p] = idx;
                const uint64_t f = fse_ring[idx];
                const uint32_t k = fcount(f);
                if (k && (int64_t)store[fstart(f)] < v) c = k;
            }
            // the lanes of one row are consecutive: one atomic per run
            const int lane = wlane();
            int first, last;
            const int sum = run_sum(v, (int)c, lane, &first, &last);
            if (ok && lane == last && sum > 0) atomicAdd(recv + v, (unsigned long long)sum);
        }
    }
}

__global__ void k_w_round(RoundCounters* ctr, uint32_t d, unsigned long long base) {
    ctr->d = d;
    ctr->cursor = base;
}

// Reset before gathering round d again into a larger store.
__global__ void k_w_rerun(RoundCounters* ctr, uint64_t* fse_new, int64_t n, unsigned long long base) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        fse_new[v] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->nO1 = ctr->nO1_base;
        ctr->nO2 = ctr->nO2_base;
        ctr->cursor = base;
        ctr->accepted = 0;
        ctr->fovf = 0;
        ctr->nU = 0;
        ctr->arcs = ctr->msgs = ctr->uniq = ctr->staged = ctr->probed = ctr->prefiltered = ctr->chk_lv = ctr->chk_lh = 0;
        ctr->tier[0] = ctr->tier[1] = ctr->tier[2] = 0;
    }
}

}  // namespace

int build_weighted_core(const int64_t* row_ptr, const int32_t* col, const uint8_t* wt, const int32_t* order,
                        int64_t n, int64_t nnz, const plb_options& o, cudaStream_t s, plb_labels** out) {
#define PLB_CK(x)                                            \
    do {                                                     \
        const cudaError_t plb_e_ = (x);                      \
        if (plb_e_ != cudaSuccess) {                         \
            (void)cudaGetLastError();                        \
            set_last_error(plb_e_, __LINE__);                \
            return PLB_ERR_CUDA;                             \
        }                                                    \
    } while (0)
#define PLB_ALLOC_OK() \
    do {               \
        if (pool.failed) return PLB_ERR_OOM; \
    } while (0)

    DevPool pool(s);
    Timer tm(o.profile != 0, s);
    const int sms = num_sms();
    const int flat_grid_cap = sms * 8;
    const int gflat = grid_for(n, kFlatThreads, flat_grid_cap);
    const int gpull = grid_for((nnz + kWTile - 1) / kWTile, 1, flat_grid_cap);
    cudaEvent_t t_all0 = tm.on ? tm.mark() : nullptr;
    int64_t launches = 0;

    int* err = pool.alloc<int>(4);
    RoundCounters* ctr = pool.alloc<RoundCounters>(1);
    PLB_ALLOC_OK();
    RoundCounters* hctr = nullptr;
    PLB_CK(cudaMallocHost(&hctr, sizeof(RoundCounters) + 4 * sizeof(int)));
    struct HostFree {
        void* p;
        ~HostFree() { cudaFreeHost(p); }
    } hf{hctr};
    int* herr = reinterpret_cast<int*>(hctr + 1);
    PLB_CK(cudaMemsetAsync(ctr, 0, sizeof(RoundCounters), s));
    PLB_CK(cudaMemsetAsync(err, 0, 4 * sizeof(int), s));

    cudaEvent_t t0 = tm.on ? tm.mark() : nullptr;
    // ------------------------------------------------- weights and validation
    // the weight range is always read: a zero weight would make a round read
    // the frontier it is writing
    const int mm_init[2] = {255, 0};
    PLB_CK(cudaMemcpyAsync(err + 2, mm_init, sizeof(mm_init), cudaMemcpyHostToDevice, s));
    if (nnz > 0) k_weight_range<<<grid_for(nnz, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(wt, nnz, err + 2);
    PLB_CK(cudaGetLastError());
    PLB_CK(cudaMemcpyAsync(herr, err, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    PLB_CK(cudaStreamSynchronize(s));
    launches += 1;
    const int minw = nnz > 0 ? herr[2] : 1, maxw = nnz > 0 ? herr[3] : 1;
    if (minw < 1) return PLB_ERR_INVALID;
    const int S = maxw + 1;  // ring slots: rounds d - maxw .. d
    // slot r mod S of the ring holds round r's descriptors at (slot << lgn) + v
    // (a power-of-two stride, so the gather reads the sender in the low bits)
    const int lgn = std::max(1, ceil_log2_i64(n));
    const int64_t ring_n = (int64_t)S << lgn;  // the empty descriptor sits at ring_n
    if (ring_n + 1 >= (int64_t(1) << 31)) return PLB_ERR_TOO_LARGE;
    if (o.validate) {
        k_check_rowptr<<<grid_for(n + 1, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(row_ptr, n, nnz, err);
        int* seen = pool.alloc<int>(n);
        PLB_ALLOC_OK();
        PLB_CK(cudaMemsetAsync(seen, 0, sizeof(int) * std::max<int64_t>(n, 1), s));
        PLB_CK(cudaMemcpyAsync(herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PLB_CK(cudaStreamSynchronize(s));
        if (herr[0]) return PLB_ERR_INVALID;
        if (nnz > 0)
            k_check_cols<<<grid_for((nnz + 2047) / 2048, 1, flat_grid_cap), kFlatThreads, 0, s>>>(row_ptr, col, n,
                                                                                               nnz, 1, err);
        k_check_order<<<grid_for(n, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(order, n, seen, err);
        PLB_CK(cudaGetLastError());
        PLB_CK(cudaMemcpyAsync(herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PLB_CK(cudaStreamSynchronize(s));
        launches += 3;
        pool.release(seen);
        if (herr[0]) return PLB_ERR_INVALID;
        if (nnz > 0) {  // arcs are symmetric and in range: compare the weights of both directions
            k_check_weights<<<grid_for((nnz + kWTile - 1) / kWTile, 1, flat_grid_cap), kWFlatThreads, 0, s>>>(
                row_ptr, col, wt, n, nnz, err);
            PLB_CK(cudaGetLastError());
            PLB_CK(cudaMemcpyAsync(herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
            PLB_CK(cudaStreamSynchronize(s));
            launches += 1;
            if (herr[0]) return PLB_ERR_INVALID;
        }
    }

    // ------------------------------------------------------- rank space
    int32_t* inv = pool.alloc<int32_t>(n);
    int64_t* roff = pool.alloc<int64_t>(n + 1);
    int32_t* rcol = pool.alloc<int32_t>(nnz);
    uint8_t* rwt = pool.alloc<uint8_t>(nnz);
    int32_t* vcol = pool.alloc<int32_t>(nnz);
    int64_t* tmp64 = pool.alloc<int64_t>(n + 1);
    int64_t* scan_scr = pool.alloc<int64_t>(scan_scratch_elems(n + 1));
    PLB_ALLOC_OK();
    const int scan_n = scan_launch_count(n);
    k_inverse<<<gflat, kFlatThreads, 0, s>>>(order, inv, n);
    k_rank_degree<<<gflat, kFlatThreads, 0, s>>>(row_ptr, order, tmp64, n);
    PLB_CK(cudaGetLastError());
    PLB_CK(exclusive_scan_i64(tmp64, roff, n, scan_scr, s));
    if (nnz > 0) {
        k_relabel<<<grid_for((nnz + 2047) / 2048, 1, flat_grid_cap), kFlatThreads, 0, s>>>(row_ptr, col, order, inv,
                                                                                          roff, rcol, n, nnz);
        k_relabel_weights<<<grid_for((nnz + kWTile - 1) / kWTile, 1, flat_grid_cap), kWFlatThreads, 0, s>>>(
            row_ptr, wt, order, roff, rwt, n, nnz);
    }
    PLB_CK(cudaGetLastError());
    launches += 4 + scan_n;

    // ------------------------------------------------------------ state
    int64_t lcap[2] = {std::max<int64_t>(2 * n, 1024), std::max<int64_t>(2 * n, 1024)};
    int64_t* loff[2] = {pool.alloc<int64_t>(n + 1), pool.alloc<int64_t>(n + 1)};
    uint32_t* lent[2] = {pool.alloc<uint32_t>(lcap[0]), pool.alloc<uint32_t>(lcap[1])};
    // frontier ring (S slots of 2^lgn descriptors, then the empty one) and store
    uint64_t* ring = pool.alloc<uint64_t>(ring_n + 1);
    int64_t scap = std::max<int64_t>(n + nnz + 1024, 4096);
    uint32_t* store = pool.alloc<uint32_t>(scap);
    uint32_t* top = pool.alloc<uint32_t>(n * kTopRow);
    int64_t* hoff = pool.alloc<int64_t>(n + 1);
    uint64_t* hdesc = pool.alloc<uint64_t>(n);
    int64_t hcap = std::max<int64_t>(4 * n, 1024);
    uint32_t* htab = pool.alloc<uint32_t>(hcap);
    unsigned long long* recv = pool.alloc<unsigned long long>(n);
    int32_t* A = pool.alloc<int32_t>(n);
    int32_t* R = pool.alloc<int32_t>(n);
    int32_t* O1 = pool.alloc<int32_t>(n);
    int32_t* U = pool.alloc<int32_t>(n);  // vertices whose new row the block tier wrote unsorted
    uint32_t* rbound = pool.alloc<uint32_t>(n);
    PLB_ALLOC_OK();
    PLB_CK(cudaMemsetAsync(ring, 0, sizeof(uint64_t) * ((size_t)ring_n + 1), s));
    PLB_CK(cudaMemsetAsync(recv, 0, sizeof(unsigned long long) * (size_t)n, s));
    // round 0: L(v) = dL_0(v) = {(v, 0)}; its frontier rows are store[0, n)
    k_init<<<gflat, kFlatThreads, 0, s>>>(roff, n, loff[0], lent[0], ring, store, A, ctr);
    k_top_init<<<flat_grid_cap, kFlatThreads, 0, s>>>(top, n);
    PLB_CK(cudaGetLastError());
    launches += 2;
    int cur = 0;
    int64_t T = n;       // labels so far
    int64_t base = n;    // store entries used (next round's rows start here)
    plb_build_stats st{};
    st.n = n;
    st.nnz = nnz;

    PLB_CK(cudaFuncSetAttribute(k_index_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(uint32_t) * kIndexWarps * kIndexSmemSlotsMax)));
    PLB_CK(cudaFuncSetAttribute(k_index_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(uint32_t) * kIndexWarps * kIndexSmemSlotsMax)));
    auto index_slots = [&](int64_t total) { return total <= 128 * n ? 512 : kIndexSmemSlotsMax; };
    auto build_index = [&]() -> int {
        if (hcap < 6 * T + 1024) {
            pool.release(htab);
            hcap = 8 * T + 1024;
            htab = pool.alloc<uint32_t>(hcap);
            if (pool.failed) return PLB_ERR_OOM;
        }
        k_index_size<<<gflat, kFlatThreads, 0, s>>>(loff[cur], n, tmp64, ctr);
        if (exclusive_scan_i64(tmp64, hoff, n, scan_scr, s) != cudaSuccess) return PLB_ERR_CUDA;
        const int slots = index_slots(T);
        k_index_build<<<grid_for((n + 255) / 256, 1, flat_grid_cap), kIndexWarps * 32,
                        sizeof(uint32_t) * kIndexWarps * slots, s>>>(loff[cur], lent[cur], hoff, htab, hdesc, n,
                                                                     slots, ctr);
        k_index_total<<<1, 1, 0, s>>>(hoff, n, ctr);
        launches += 3 + scan_n;
        return cudaGetLastError() == cudaSuccess ? PLB_OK : PLB_ERR_CUDA;
    };
    {
        const int e = build_index();
        if (e != PLB_OK) return e;
    }
    if (tm.on) tm.span(T_PREP, t0, tm.mark());

    // tier geometry (as in the undirected build)
    const int warp_cand = pow2_at_least(std::max(32, o.warp_cand_cap));
    const int warp_label = std::max(16, o.warp_label_cap);
    const int w_log_s = ceil_log2_i64(std::max<int64_t>(2 * warp_cand, warp_cand + 32 * kGatherUnroll));
    const int w_log_m = ceil_log2_i64(2 * warp_label);
    const int warps_per_block = kGpWarpThreads / 32;
    const size_t w_smem = sizeof(uint32_t) * (4 * warps_per_block +
                                              (size_t)warps_per_block * (kTopRow + (1 << w_log_s) + (1 << w_log_m)));
    const int bthr = std::min(256, std::max(64, (o.block_threads / 32) * 32));
    const int block_cand = pow2_at_least(std::max(bthr, o.block_cand_cap));
    const int b_log_s = ceil_log2_i64(std::max<int64_t>(
        std::max<int64_t>(2 * (int64_t)block_cand, block_cand + (int64_t)kGatherUnroll * bthr),
        (int64_t)kByteStage * (bthr / 32)));
    const int b_log_m = ceil_log2_i64(2 * (int64_t)std::max(o.block_label_cap, 64) + 2 * bthr);
    const size_t b_smem = gp_block_smem_bytes(bthr, b_log_s, b_log_m, block_cand);
    TierLimits lim;
    lim.warp_bound = 2 * (int64_t)warp_cand;
    lim.warp_label = warp_label;
    lim.warp_deg = (int64_t)32 * 64;
    if (w_smem > 227 * 1024 || b_smem > 227 * 1024) return PLB_ERR_INVALID;
    PLB_CK(cudaFuncSetAttribute(k_gp_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w_smem));
    PLB_CK(cudaFuncSetAttribute(k_gp_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b_smem));
    PLB_CK(cudaFuncSetAttribute(k_sort_rows_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(16384 * sizeof(uint32_t))));
    int occ_w = 1, occ_b = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_w, k_gp_warp, kGpWarpThreads, w_smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, k_gp_block, bthr, b_smem);
    const int grid_w = sms * std::max(1, occ_w);
    const int grid_b = sms * std::max(1, occ_b);
    int32_t* big = pool.alloc<int32_t>(n);
    int32_t* giant = pool.alloc<int32_t>(n);
    const int sort_blocks = 8;
    const int64_t sort_words = pow2_at_least(std::max<int64_t>(n, 1));
    uint32_t* sortscr = pool.alloc<uint32_t>(sort_words * sort_blocks);
    uint32_t* gacc = pool.alloc<uint32_t>((int64_t)grid_b * std::max<int64_t>(n, 1));
    PLB_ALLOC_OK();

    auto read_ctr = [&]() -> cudaError_t {
        return cudaMemcpyAsync(hctr, ctr, sizeof(RoundCounters), cudaMemcpyDeviceToHost, s);
    };
    // grow the store to hold `need` entries, keeping every row at its offset
    auto grow_store = [&](int64_t need) -> int {
        const int64_t ncap = std::max<int64_t>(need + need / 4 + 1024, 2 * scap);
        uint32_t* ns = pool.alloc<uint32_t>(ncap);
        if (pool.failed) return PLB_ERR_OOM;
        if (base > 0 && cudaMemcpyAsync(ns, store, sizeof(uint32_t) * base, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return PLB_ERR_CUDA;
        pool.release(store);
        store = ns;
        scap = ncap;
        return PLB_OK;
    };
    auto gather = [&](uint64_t* fse_new) -> cudaError_t {
        GpParams p{};
        p.roff = roff;
        p.rcol = vcol;
        p.loff = loff[cur];
        p.lent = lent[cur];
        p.fse = ring;
        p.fhub = store;
        p.fse_new = fse_new;
        p.fhub_new = store;
        p.fcap = (unsigned long long)scap;
        p.ctr = ctr;
        p.hdesc = hdesc;
        p.htab = htab;
        p.top = top;
        p.loff_h = loff[cur];
        p.lent_h = lent[cur];
        p.hdesc_h = hdesc;
        p.htab_h = htab;
        p.top_h = top;
        p.gscratch = gacc;
        p.gscratch_words = std::max<int64_t>(n, 1);
        p.rbound = rbound;
        p.ostart = nullptr;
        p.sender_bits = lgn;
        p.list = R;
        p.list_n = &ctr->nR;
        p.esc = O1;
        p.esc_n = &ctr->nO1;
        p.log_s = w_log_s;
        p.log_m = w_log_m;
        p.cand_limit = warp_cand;
        p.stage_ratio = o.warp_stage_ratio;
        p.count_check = o.profile != 0;
        p.unsorted = U;
        k_gp_warp<<<grid_w, kGpWarpThreads, w_smem, s>>>(p);
        p.list = O1;
        p.list_n = &ctr->nO1;
        p.esc = nullptr;
        p.esc_n = nullptr;
        p.log_s = b_log_s;
        p.log_m = b_log_m;
        p.cand_limit = block_cand;
        k_gp_block<<<grid_b, bthr, b_smem, s>>>(p);
        launches += 2;
        return cudaGetLastError();
    };

    // ------------------------------------------------------------ rounds
    int status = PLB_OK;
    int last = 0;  // last round that accepted labels (round 0: the self labels)
    int rounds = 0;
    for (int d = 1; d - last <= maxw; ++d) {
        uint64_t* fse_new = ring + ((int64_t)(d % S) << lgn);
        cudaEvent_t r0 = tm.on ? tm.mark() : nullptr;
        k_w_round<<<1, 1, 0, s>>>(ctr, (uint32_t)d, (unsigned long long)base);
        if (nnz > 0)
            k_w_pull<<<gpull, kWFlatThreads, 0, s>>>(roff, rcol, rwt, n, nnz, (uint32_t)d, S, lgn, ring, store,
                                                     vcol, recv);
        k_collect<<<gflat, kFlatThreads, 0, s>>>(recv, roff, loff[cur], n, fse_new, R, O1, rbound, nullptr, ctr, lim);
        k_after_collect<<<1, 1, 0, s>>>(ctr);
        launches += 4;
        PLB_CK(cudaGetLastError());
        PLB_CK(read_ctr());
        PLB_CK(cudaStreamSynchronize(s));
        if (hctr->hovf) {
            const int e = build_index();
            if (e != PLB_OK) return e;
        }
        if (base + (int64_t)hctr->bound_sum > scap) {
            const int e = grow_store(base + (int64_t)hctr->bound_sum);
            if (e != PLB_OK) return e;
        }
        if (tm.on) tm.span(T_FRONT, r0, tm.mark());
        cudaEvent_t g0 = tm.on ? tm.mark() : nullptr;
        const bool any = hctr->nR + hctr->nO1_base > 0;
        if (any) {
            for (int attempt = 0;; ++attempt) {
                if (attempt > 0) {
                    k_w_rerun<<<gflat, kFlatThreads, 0, s>>>(ctr, fse_new, n, (unsigned long long)base);
                    launches += 1;
                }
                PLB_CK(gather(fse_new));
                PLB_CK(read_ctr());
                PLB_CK(cudaStreamSynchronize(s));
                if (hctr->guard) return PLB_ERR_CUDA;
                if (!hctr->fovf) break;
                if (attempt >= 4) return PLB_ERR_CUDA;  // the bound above covers every row
                const int e = grow_store((int64_t)hctr->cursor);
                if (e != PLB_OK) return e;
                st.reruns += 1;
            }
        }
        if (tm.on) tm.span(T_GPW, g0, tm.mark());
        const int64_t acc = any ? (int64_t)hctr->accepted : 0;
        if (d < PLB_MAX_ROUNDS) {
            st.receivers[d] = (int64_t)hctr->nR + hctr->nO1_base;
            st.accepted[d] = acc;
            st.unique_round[d] = any ? (int64_t)hctr->uniq : 0;
            st.prefiltered_round[d] = any ? (int64_t)hctr->prefiltered : 0;
            st.probed_round[d] = any ? (int64_t)hctr->probed : 0;
            st.messages_round[d] = any ? (int64_t)hctr->msgs : 0;
        }
        if (any) {
            st.arcs_scanned += (int64_t)hctr->arcs;
            st.messages += (int64_t)hctr->msgs;
            st.unique_candidates += (int64_t)hctr->uniq;
            st.staged_entries += (int64_t)hctr->staged;
            st.probed_entries += (int64_t)hctr->probed;
            st.check_lv_entries += (int64_t)hctr->chk_lv;
            st.check_lh_entries += (int64_t)hctr->chk_lh;
            for (int q = 0; q < 3; ++q) st.tier_vertices[q] += (int64_t)hctr->tier[q];
        }
        rounds = d;
        if (acc > 0) {
            if (d > PLB_MAX_DIST) {
                status = PLB_ERR_DIST_OVERFLOW;
                break;
            }
            last = d;
            // merge dL_d into L (rows sorted by hub rank) and index it
            cudaEvent_t m0 = tm.on ? tm.mark() : nullptr;
            const int x = cur ^ 1;
            const int64_t Tn = T + acc;
            if (Tn > lcap[x]) {
                pool.release(lent[x]);
                lcap[x] = Tn + Tn / 4 + 1024;
                lent[x] = pool.alloc<uint32_t>(lcap[x]);
                PLB_ALLOC_OK();
            }
            k_next_active<<<gflat, kFlatThreads, 0, s>>>(loff[cur], fse_new, n, tmp64, A, ctr);
            k_sort_rows_warp<<<sms * 8, 256, 0, s>>>(fse_new, store, A, U, 0, ctr, big, giant);
            k_sort_rows_block<<<sms * 2, 1024, 16384 * sizeof(uint32_t), s>>>(fse_new, store, big, &ctr->nBig,
                                                                            nullptr, 0, ctr);
            k_sort_rows_block<<<sort_blocks, 1024, 16384 * sizeof(uint32_t), s>>>(fse_new, store, giant,
                                                                                &ctr->nGiant, sortscr, sort_words,
                                                                                ctr);
            PLB_CK(exclusive_scan_i64(tmp64, loff[x], n, scan_scr, s));
            k_merge_old<<<flat_grid_cap, kFlatThreads, 0, s>>>(loff[cur], lent[cur], loff[x], lent[x], fse_new, store,
                                                               n, ctr);
            k_merge_new<<<grid_for((int64_t)n * 32, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(
                loff[cur], lent[cur], loff[x], lent[x], fse_new, store, A, ctr, top);
            launches += 6 + scan_n;
            PLB_CK(cudaGetLastError());
            const int64_t Told = T;
            T = Tn;
            cur = x;
            if (acc > Told) {  // more than doubles the labels: most tables outgrown, repack
                const int e = build_index();
                if (e != PLB_OK) return e;
            } else {
                const int slots = index_slots(Tn);
                k_index_update<<<flat_grid_cap, kIndexWarps * 32, sizeof(uint32_t) * kIndexWarps * slots, s>>>(
                    loff[x], lent[x], fse_new, store, A, htab, hdesc, (long long)hcap, slots, ctr);
                launches += 1;
                PLB_CK(cudaGetLastError());
            }
            base = (int64_t)hctr->cursor;  // this round's rows end here
            if (tm.on) tm.span(T_MERGE, m0, tm.mark());
        }
        PLB_CK(cudaMemsetAsync(ctr, 0, offsetof(RoundCounters, nA), s));
        PLB_CK(cudaMemsetAsync(&ctr->nO1_base, 0, sizeof(int) * 3, s));
    }
    if (status != PLB_OK) return status;

    // ------------------------------------------------------------ finalize
    // the round buffers go back to the pool before the label set is allocated
    pool.release_all_except({loff[cur], lent[cur], inv, tmp64, scan_scr, ctr});
    cudaEvent_t f0 = tm.on ? tm.mark() : nullptr;
    plb_labels* L = new plb_labels();
    auto fail = [&](int code) {
        if (L->off) cudaFreeAsync(L->off, s);
        if (L->packed) cudaFreeAsync(L->packed, s);
        if (L->hub) cudaFreeAsync(L->hub, s);
        if (L->dist) cudaFreeAsync(L->dist, s);
        if (L->order) cudaFreeAsync(L->order, s);
        delete L;
        return code;
    };
    L->n = n;
    L->total = T;
    L->rounds = rounds;
    if (plb::dev_alloc((void**)&L->off, sizeof(int64_t) * (n + 1), s) != cudaSuccess ||
        plb::dev_alloc((void**)&L->packed, sizeof(uint32_t) * std::max<int64_t>(T, 1), s) != cudaSuccess ||
        plb::dev_alloc((void**)&L->hub, sizeof(uint32_t) * std::max<int64_t>(T, 1), s) != cudaSuccess ||
        plb::dev_alloc((void**)&L->dist, std::max<int64_t>(T, 1), s) != cudaSuccess ||
        plb::dev_alloc((void**)&L->order, sizeof(int32_t) * std::max<int64_t>(n, 1), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(PLB_ERR_OOM);
    }
    L->bytes = (int64_t)(sizeof(int64_t) * (n + 1) + 9 * (size_t)T + 4 * (size_t)n);
    k_final_len<<<gflat, kFlatThreads, 0, s>>>(loff[cur], inv, n, tmp64);
    if (exclusive_scan_i64(tmp64, L->off, n, scan_scr, s) != cudaSuccess) return fail(PLB_ERR_CUDA);
    k_finalize<<<grid_for((T + 2047) / 2048, 1, flat_grid_cap), kFlatThreads, 0, s>>>(
        loff[cur], lent[cur], inv, L->off, L->packed, L->hub, L->dist, n, ctr);
    if (cudaMemcpyAsync(L->order, order, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        read_ctr() != cudaSuccess)
        return fail(PLB_ERR_CUDA);
    launches += 2 + scan_n;
    cudaEvent_t f1 = tm.on ? tm.mark() : nullptr;
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(PLB_ERR_CUDA);
    L->max_dist = (int32_t)hctr->max_dist;
    st.rounds = rounds;
    st.total_labels = T;
    st.launches = launches;
    if (tm.on) {
        tm.span(T_FINAL, f0, f1);
        tm.span(T_ALL, t_all0, f1);
        st.ms_prepare = tm.total(T_PREP);
        st.ms_frontier = tm.total(T_FRONT);
        st.ms_gather_prune[0] = tm.total(T_GPW);
        st.ms_merge = tm.total(T_MERGE);
        st.ms_finalize = tm.total(T_FINAL);
        st.ms_total = tm.total(T_ALL);
    }
    L->stats = st;
    *out = L;
    return PLB_OK;
#undef PLB_CK
#undef PLB_ALLOC_OK
}

}  // namespace plb
