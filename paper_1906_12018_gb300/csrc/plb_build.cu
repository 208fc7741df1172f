// Host driver of the labeling build: validation, rank-space relabel, the
// round loop of Alg. 3 (Sec. 3.1) and the final by-id label layout.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <vector>

#include "plb_host.cuh"

namespace plb {

thread_local char g_last_error[256] = "";

void set_last_error(cudaError_t e, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "plb_build.cu:%d: %s (%s)", line, cudaGetErrorString(e),
             cudaGetErrorName(e));
}

// Core build on a validated-or-trusted CSR.  Returns a status; on success
// *out holds the labels (rows by original id).  max_part_n: the most vertices
// of one graph when the CSR is a disjoint union (else n); a vertex's label
// holds at most that many hubs, which sizes the block tier's accepted rows.
int build_core(const int64_t* row_ptr, const int32_t* col, const int32_t* order, int64_t n, int64_t nnz,
               const plb_options& o, cudaStream_t s, plb_labels** out, int64_t max_part_n) {
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
    plb_build_stats st{};
    st.n = n;
    st.nnz = nnz;
    const int sms = num_sms();
    const int flat_grid_cap = sms * 8;
    cudaEvent_t t_all0 = tm.on ? tm.mark() : nullptr;

    RoundCounters* ctr = pool.alloc<RoundCounters>(1);
    int* err = pool.alloc<int>(4);
    PLB_ALLOC_OK();
    RoundCounters* hctr = nullptr;
    PLB_CK(cudaMallocHost(&hctr, sizeof(RoundCounters)));
    struct HostFree {
        void* p;
        ~HostFree() { cudaFreeHost(p); }
    } hf{hctr};
    PLB_CK(cudaMemsetAsync(ctr, 0, sizeof(RoundCounters), s));
    PLB_CK(cudaMemsetAsync(err, 0, 4 * sizeof(int), s));

    cudaEvent_t t0 = tm.on ? tm.mark() : nullptr;
    // ---------------------------------------------------------- validation
    if (o.validate) {
        k_check_rowptr<<<grid_for(n + 1, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(row_ptr, n, nnz, err);
        PLB_CK(cudaGetLastError());
        int herr = 0;
        PLB_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PLB_CK(cudaStreamSynchronize(s));
        st.launches += 1;
        if (herr) return PLB_ERR_INVALID;
        int* seen = pool.alloc<int>(n);
        PLB_ALLOC_OK();
        PLB_CK(cudaMemsetAsync(seen, 0, sizeof(int) * std::max<int64_t>(n, 1), s));
        if (nnz > 0) {
            k_check_cols<<<grid_for((nnz + 2047) / 2048, 1, flat_grid_cap), kFlatThreads, 0, s>>>(row_ptr, col, n,
                                                                                               nnz, 1, err);
            PLB_CK(cudaGetLastError());
        }
        k_check_order<<<grid_for(n, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(order, n, seen, err);
        PLB_CK(cudaGetLastError());
        PLB_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PLB_CK(cudaStreamSynchronize(s));
        st.launches += 2;
        pool.release(seen);
        if (herr) return PLB_ERR_INVALID;
    }

    // ---------------------------------------------------- rank-space CSR
    int32_t* inv = pool.alloc<int32_t>(n);
    int64_t* roff = pool.alloc<int64_t>(n + 1);
    int32_t* rcol = pool.alloc<int32_t>(nnz);
    int64_t* tmp64 = pool.alloc<int64_t>(n + 1);
    int64_t* scan_scr = pool.alloc<int64_t>(scan_scratch_elems(n + 1));
    PLB_ALLOC_OK();
    const int gflat = grid_for(n, kFlatThreads, flat_grid_cap);
    k_inverse<<<gflat, kFlatThreads, 0, s>>>(order, inv, n);
    k_rank_degree<<<gflat, kFlatThreads, 0, s>>>(row_ptr, order, tmp64, n);
    PLB_CK(cudaGetLastError());
    PLB_CK(exclusive_scan_i64(tmp64, roff, n, scan_scr, s));
    if (nnz > 0) {
        k_relabel<<<grid_for((nnz + 2047) / 2048, 1, flat_grid_cap), kFlatThreads, 0, s>>>(row_ptr, col, order, inv,
                                                                                          roff, rcol, n, nnz);
        PLB_CK(cudaGetLastError());
    }
    st.launches += 3 + scan_launch_count(n);
    const int scan_n = scan_launch_count(n);  // launches of one scan over n values

    // ------------------------------------------------------------ state
    int64_t lcap[2] = {std::max<int64_t>(2 * n, 1024), std::max<int64_t>(2 * n, 1024)};
    int64_t* loff[2] = {pool.alloc<int64_t>(n + 1), pool.alloc<int64_t>(n + 1)};
    uint32_t* lent[2] = {pool.alloc<uint32_t>(lcap[0]), pool.alloc<uint32_t>(lcap[1])};
    int64_t fcap[2] = {std::max<int64_t>(nnz / 2 + n, 1024), std::max<int64_t>(nnz / 2 + n, 1024)};
    uint64_t* fse[2] = {pool.alloc<uint64_t>(n), pool.alloc<uint64_t>(n)};
    uint32_t* fhub[2] = {pool.alloc<uint32_t>(fcap[0]), pool.alloc<uint32_t>(fcap[1])};
    unsigned long long* recv = pool.alloc<unsigned long long>(n);
    int32_t* A = pool.alloc<int32_t>(n);
    int32_t* R = pool.alloc<int32_t>(n);
    int32_t* O1 = pool.alloc<int32_t>(n);
    int32_t* O2 = pool.alloc<int32_t>(n);  // warp-tier escalations when the two tiers run concurrently
    uint32_t* rbound = pool.alloc<uint32_t>(n);
    uint32_t* cur1 = pool.alloc<uint32_t>(n);  // round 1: per-row write cursors
    int32_t* U = pool.alloc<int32_t>(n);       // vertices whose new row the block tier wrote unsorted
    int64_t* aoff = pool.alloc<int64_t>(n + 1);
    PLB_ALLOC_OK();
    PLB_CK(cudaMemsetAsync(recv, 0, sizeof(unsigned long long) * std::max<int64_t>(n, 1), s));
    k_init<<<gflat, kFlatThreads, 0, s>>>(roff, n, loff[0], lent[0], fse[0], fhub[0], A, ctr);
    PLB_CK(cudaGetLastError());
    st.launches += 1;
    int64_t T = n;  // labels so far
    int cur = 0;    // index of current L and previous frontier
    // top-hub distance rows (witness prefilter), updated by each merge
    uint32_t* top = pool.alloc<uint32_t>(n * kTopRow);
    PLB_ALLOC_OK();
    k_top_init<<<flat_grid_cap, kFlatThreads, 0, s>>>(top, n);
    st.launches += 1;
    // probe index of L: a hub-keyed table per row of >= kIndexMinLen entries in
    // a pool (htab), located by hdesc.  A full rebuild packs the tables and
    // leaves room for growth; after each merge only the rows that changed are
    // updated (new entries inserted, or a bigger table taken from the pool).
    int64_t* hoff = pool.alloc<int64_t>(n + 1);
    uint64_t* hdesc = pool.alloc<uint64_t>(n);
    int64_t hcap = std::max<int64_t>(4 * n, 1024);
    uint32_t* htab = pool.alloc<uint32_t>(hcap);
    PLB_ALLOC_OK();
    PLB_CK(cudaFuncSetAttribute(k_index_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(uint32_t) * kIndexWarps * kIndexSmemSlotsMax)));
    PLB_CK(cudaFuncSetAttribute(k_index_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(uint32_t) * kIndexWarps * kIndexSmemSlotsMax)));
    // shared-memory table buffer of the index kernels: 512 slots while the mean
    // row is short (most tables fit and eight blocks share an SM), else 2048
    auto index_slots = [&](int64_t total) { return total <= 128 * n ? 512 : kIndexSmemSlotsMax; };
    // Table pool size.  roomy: from the bound (packed tables take at most
    // 4 |L| slots; as much again for growth), for graph segments whose rounds
    // all update the index in place.  Otherwise from the packed tables' exact
    // slot count (hoff[n], read back), with half as much again for the
    // in-place updates of the following rounds; a pool that still overflows
    // is repacked before the next gather.
    auto build_index = [&](int which, int64_t total, bool roomy) -> int {
        k_index_size<<<gflat, kFlatThreads, 0, s>>>(loff[which], n, tmp64, ctr);
        if (exclusive_scan_i64(tmp64, hoff, n, scan_scr, s) != cudaSuccess) return PLB_ERR_CUDA;
        int64_t need = 6 * total + 1024, want = 8 * total + 1024;
        if (!roomy) {
            int64_t packed = 0;
            int done = 0;
            if (cudaMemcpyAsync(&packed, hoff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(&done, &ctr->done, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return PLB_ERR_CUDA;
            if (done) return PLB_OK;  // a finished build: the index kernels would return at once
            need = packed + 1024;
            want = packed + packed / 2 + 1024;
        }
        if (hcap < need || (!roomy && hcap > 2 * want)) {
            pool.release(htab);
            hcap = want;
            htab = pool.alloc<uint32_t>(hcap);
            if (pool.failed) return PLB_ERR_OOM;
        }
        const int slots = index_slots(total);
        k_index_build<<<grid_for((n + 255) / 256, 1, flat_grid_cap), kIndexWarps * 32,
                        sizeof(uint32_t) * kIndexWarps * slots, s>>>(loff[which], lent[which], hoff, htab, hdesc, n,
                                                                     slots, ctr);
        k_index_total<<<1, 1, 0, s>>>(hoff, n, ctr);
        st.launches += 3 + scan_n;
        return cudaGetLastError() == cudaSuccess ? PLB_OK : PLB_ERR_CUDA;
    };
    // after a merge into parity c (labels and this round's frontier): update the
    // rows that changed (the active list)
    auto update_index = [&](int c, int64_t total) -> cudaError_t {
        const int slots = index_slots(total);
        k_index_update<<<flat_grid_cap, kIndexWarps * 32, sizeof(uint32_t) * kIndexWarps * slots, s>>>(
            loff[c], lent[c], fse[c], fhub[c], A, htab, hdesc, (long long)hcap, slots, ctr);
        st.launches += 1;
        return cudaGetLastError();
    };
    {
        const int e = build_index(0, T, false);
        if (e != PLB_OK) return e;
    }
    if (tm.on) tm.span(T_PREP, t0, tm.mark());

    // tier geometry
    const int warp_cand = pow2_at_least(std::max(32, o.warp_cand_cap));
    const int warp_label = std::max(16, o.warp_label_cap);
    // set tables: load <= 1/2 at the candidate limit, plus the inserts a gather
    // step can make before it sees the count (kGatherUnroll x 32 per warp)
    const int w_log_s = ceil_log2_i64(std::max<int64_t>(2 * warp_cand, warp_cand + 32 * kGatherUnroll));
    const int w_log_m = ceil_log2_i64(2 * warp_label);
    const int warps_per_block = kGpWarpThreads / 32;
    const size_t w_smem = sizeof(uint32_t) * (4 * warps_per_block +
                                              (size_t)warps_per_block * (kTopRow + (1 << w_log_s) + (1 << w_log_m)));
    const int bthr = std::min(256, std::max(64, (o.block_threads / 32) * 32));  // k_gp_block: <= 256 threads
    const int block_cand = pow2_at_least(std::max(bthr, o.block_cand_cap));
    const int b_log_s = ceil_log2_i64(std::max<int64_t>(std::max<int64_t>(2 * (int64_t)block_cand,
                                                                           block_cand + (int64_t)kGatherUnroll * bthr),
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
    int occ_w = 1, occ_b = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_w, k_gp_warp, kGpWarpThreads, w_smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, k_gp_block, bthr, b_smem);
    const int grid_w = sms * std::max(1, occ_w);
    const int grid_b = sms * std::max(1, occ_b);
    // long frontier rows: block-per-row sort (power-of-two scratch per block)
    int32_t* big = pool.alloc<int32_t>(n);
    int32_t* giant = pool.alloc<int32_t>(n);
    const int sort_blocks = 8;
    const int64_t sort_words = pow2_at_least(std::max<int64_t>(n, 1));
    uint32_t* sortscr = pool.alloc<uint32_t>(sort_words * sort_blocks);
    PLB_ALLOC_OK();
    PLB_CK(cudaFuncSetAttribute(k_sort_rows_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(16384 * sizeof(uint32_t))));
    PLB_CK(cudaFuncSetAttribute(k_sort_rows_radix, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortRadixSmemBytes));
    // block tier: per-block buffer of accepted hubs (at most v < n per vertex)
    const int64_t acc_words = std::max<int64_t>(std::min<int64_t>(n, max_part_n), 1);
    uint32_t* gacc = pool.alloc<uint32_t>((int64_t)grid_b * acc_words);
    // per-vertex check records (row bounds and probe-table descriptor), packed before each gather
    uint4* hrec = pool.alloc<uint4>(std::max<int64_t>(n, 1));
    PLB_ALLOC_OK();

    // ------------------------------------------------------------ rounds
    // launch sequences of one round (buffers of parity c -> x = c ^ 1)
    // placed: the new-frontier buffer holds the bound sum, so the rows go where
    // the scan of the bounds (aoff, after the frontier step) puts them
    auto gp_params = [&](int c, int x, int64_t fc, bool placed) {
        GpParams p{};
        p.ostart = placed ? aoff : nullptr;
        p.roff = roff;
        p.rcol = rcol;
        p.loff = loff[c];
        p.lent = lent[c];
        p.fse = fse[c];
        p.fhub = fhub[c];
        p.fse_new = fse[x];
        p.fhub_new = fhub[x];
        p.fcap = (unsigned long long)fc;
        p.ctr = ctr;
        p.hdesc = hdesc;
        p.htab = htab;
        p.loff_h = loff[c];
        p.lent_h = lent[c];
        p.hdesc_h = hdesc;
        p.htab_h = htab;
        p.top = top;
        p.top_h = top;
        p.hrec_h = hrec;
        p.gscratch = gacc;
        p.gscratch_words = acc_words;
        p.rbound = rbound;
        p.stage_ratio = o.warp_stage_ratio;
        p.count_check = o.profile != 0;
        p.unsorted = U;
        return p;
    };
    const int* skip = nullptr;  // graph mode: &ctr->done (scans of finished rounds do nothing)
    auto launch_frontier = [&](int c, int x) -> cudaError_t {
        k_active_degree<<<gflat, kFlatThreads, 0, s>>>(roff, A, ctr, tmp64, n);
        cudaError_t e = exclusive_scan_i64(tmp64, aoff, n, scan_scr, s, skip);
        if (e != cudaSuccess) return e;
        k_mark<<<flat_grid_cap, kFlatThreads, 0, s>>>(roff, rcol, fse[c], fhub[c], A, aoff, ctr, recv, n);
        k_collect<<<gflat, kFlatThreads, 0, s>>>(recv, roff, loff[c], n, fse[x], R, O1, rbound, tmp64, ctr, lim);
        k_after_collect<<<1, 1, 0, s>>>(ctr);
        // the scan of the candidate bounds places each receiver's new frontier
        // row (aoff is free again after k_mark); used when the buffer holds
        // the bound sum, so that no shared cursor is contended
        e = exclusive_scan_i64(tmp64, aoff, n, scan_scr, s, skip);
        if (e != cudaSuccess) return e;
        st.launches += 4 + 2 * scan_n;
        return cudaGetLastError();
    };
    // Host-driven rounds run the two tiers concurrently: the block tier on a
    // side stream over k_collect's block list while the warp tier runs on the
    // build's stream and escalates into a second list, taken by one more
    // block-tier launch after both (the tails of the two kernels overlap).
    // Captured rounds (graph mode) run them one after the other.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    PLB_CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    PLB_CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    PLB_CK(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
    struct SideGuard {
        cudaStream_t st;
        cudaEvent_t a, b;
        ~SideGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            cudaStreamDestroy(st);
        }
    } side_guard{side, ev_fork, ev_join};
    auto launch_gp = [&](GpParams p, cudaEvent_t* g1) -> cudaError_t {
        k_pack_hrec<<<gflat, kFlatThreads, 0, s>>>(p.loff, p.lent, hdesc, hrec, n, ctr);
        st.launches += 1;
        GpParams w = p, b = p;
        w.list = R;  // warp tier
        w.list_n = &ctr->nR;
        w.log_s = w_log_s;
        w.log_m = w_log_m;
        w.cand_limit = warp_cand;
        b.esc = nullptr;  // block tier (never escalates)
        b.esc_n = nullptr;
        b.log_s = b_log_s;
        b.log_m = b_log_m;
        b.cand_limit = block_cand;
        if (skip == nullptr) {
            w.esc = O2;
            w.esc_n = &ctr->nO2;
            b.list = O1;
            b.list_n = &ctr->nO1;
            cudaError_t e = cudaEventRecord(ev_fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_fork, 0);
            if (e != cudaSuccess) return e;
            k_gp_block<<<grid_b, bthr, b_smem, side>>>(b);
            k_gp_warp<<<grid_w, kGpWarpThreads, w_smem, s>>>(w);
            if (g1) *g1 = tm.mark();
            e = cudaEventRecord(ev_join, side);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_join, 0);
            if (e != cudaSuccess) return e;
            b.list = O2;
            b.list_n = &ctr->nO2;
            k_gp_block<<<grid_b, bthr, b_smem, s>>>(b);
            st.launches += 3;
            return cudaGetLastError();
        }
        w.esc = O1;
        w.esc_n = &ctr->nO1;
        k_gp_warp<<<grid_w, kGpWarpThreads, w_smem, s>>>(w);
        if (g1) *g1 = tm.mark();
        b.list = O1;
        b.list_n = &ctr->nO1;
        k_gp_block<<<grid_b, bthr, b_smem, s>>>(b);
        st.launches += 2;
        return cudaGetLastError();
    };
    auto launch_merge = [&](int c, int x) -> cudaError_t {
        k_next_active<<<gflat, kFlatThreads, 0, s>>>(loff[c], fse[x], n, tmp64, A, ctr);
        // sort the new frontier rows (appended unsorted by the gather/prune kernels)
        k_sort_rows_warp<<<sms * 8, 256, 0, s>>>(fse[x], fhub[x], A, U, 1, ctr, big, giant);
        k_sort_rows_radix<<<sms, 1024, kSortRadixSmemBytes, s>>>(fse[x], fhub[x], big, &ctr->nBig, ctr);
        k_sort_rows_block<<<sort_blocks, 1024, 16384 * sizeof(uint32_t), s>>>(fse[x], fhub[x], giant, &ctr->nGiant,
                                                                            sortscr, sort_words, ctr);
        cudaError_t e = exclusive_scan_i64(tmp64, loff[x], n, scan_scr, s, skip);
        if (e != cudaSuccess) return e;
        k_merge_old<<<flat_grid_cap, kFlatThreads, 0, s>>>(loff[c], lent[c], loff[x], lent[x], fse[x], fhub[x], n,
                                                           ctr);
        k_merge_new<<<grid_for((int64_t)n * 32, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(
            loff[c], lent[c], loff[x], lent[x], fse[x], fhub[x], A, ctr, top);
        st.launches += 6 + scan_n;
        return cudaGetLastError();
    };

    int status = PLB_OK;
    int d = 0;          // last completed round (of the current batch)
    bool finished = false;
    // hubs of the current batch (Alg. 4): ranks [batch_lo, batch_hi); one batch
    // of all vertices is Alg. 3
    const int64_t batch = o.batch_hubs > 0 ? std::min<int64_t>(o.batch_hubs, n) : n;
    int64_t batch_lo = 0, batch_hi = n;
    std::vector<std::pair<int, cudaEvent_t>> round_ev;  // (round, start event)
    std::vector<char> host_stat(PLB_MAX_ROUNDS, 0);     // rounds whose statistics the host recorded

    // One host-driven round (d + 1).  With frontier_done the round's frontier
    // step has already run (a graph stopped after it) and ctr->d holds d + 1.
    auto host_round = [&](bool frontier_done) -> int {
        ++d;
        const int nxt = cur ^ 1;
        cudaEvent_t r0 = tm.on ? tm.mark() : nullptr;
        if (d == 1) {
            // round 1 needs no frontier step and no check (k_round1); the
            // new-frontier buffer holds every arc
            k_set_round<<<1, 1, 0, s>>>(ctr, 1u);
            const int g1 = grid_for((nnz + 2047) / 2048, 1, flat_grid_cap);
            PLB_CK(cudaMemsetAsync(tmp64, 0, sizeof(int64_t) * (n + 1), s));
            PLB_CK(cudaMemsetAsync(cur1, 0, sizeof(uint32_t) * std::max<int64_t>(n, 1), s));
            if (nnz > 0)
                k_round1_count<<<g1, kFlatThreads, 0, s>>>(roff, rcol, n, nnz, (int32_t)batch_lo, (int32_t)batch_hi,
                                                          reinterpret_cast<unsigned long long*>(tmp64), ctr);
            PLB_CK(exclusive_scan_i64(tmp64, tmp64, n, scan_scr, s));
            k_round1<<<g1, kFlatThreads, 0, s>>>(roff, rcol, n, nnz, (int32_t)batch_lo, (int32_t)batch_hi, tmp64,
                                                cur1, fse[nxt], fhub[nxt], (unsigned long long)fcap[nxt], ctr);
            st.launches += 3 + scan_n;
            PLB_CK(cudaGetLastError());
            PLB_CK(cudaMemcpyAsync(hctr, ctr, sizeof(RoundCounters), cudaMemcpyDeviceToHost, s));
            PLB_CK(cudaStreamSynchronize(s));
            if (hctr->fovf) return PLB_ERR_CUDA;
            if (tm.on) {
                cudaEvent_t r1 = tm.mark();
                tm.span(T_GPW, r0, r1);
            }
        } else {
            if (!frontier_done) {
                k_set_round<<<1, 1, 0, s>>>(ctr, (uint32_t)d);
                st.launches += 1;
                // frontier: mark receivers from the active list, collect them
                PLB_CK(launch_frontier(cur, nxt));
            }
            // size the new frontier buffer from the candidate bound (no re-run)
            PLB_CK(cudaMemcpyAsync(hctr, ctr, sizeof(RoundCounters), cudaMemcpyDeviceToHost, s));
            PLB_CK(cudaStreamSynchronize(s));
            if (hctr->hovf) {  // the last update did not fit the table pool: rebuild it, packed
                const int e = build_index(cur, T, false);
                if (e != PLB_OK) return e;
            }
            // (up to 2^31 entries: past that the buffer holds twice the last
            // round's acceptance, set after the merge, and a round that still
            // overflows it runs again; the bound far exceeds the acceptance of
            // the rounds after the largest)
            if ((int64_t)hctr->bound_sum > fcap[nxt]) {
                const int64_t want = std::min<int64_t>((int64_t)hctr->bound_sum + 1024,
                                                       std::max<int64_t>(int64_t(1) << 31, fcap[nxt]));
                if (want > fcap[nxt]) {
                    pool.release(fhub[nxt]);
                    fcap[nxt] = want;
                    fhub[nxt] = pool.alloc<uint32_t>(fcap[nxt]);
                    PLB_ALLOC_OK();
                }
            }
            cudaEvent_t r1 = tm.on ? tm.mark() : nullptr;
            if (tm.on) tm.span(T_FRONT, r0, r1);
            bool rerun = false;
            for (;;) {
                if (rerun) {
                    k_rerun_reset<<<gflat, kFlatThreads, 0, s>>>(ctr, fse[nxt], n);
                    st.launches += 1;
                }
                cudaEvent_t g0 = tm.on ? tm.mark() : nullptr, g1 = nullptr;
                PLB_CK(launch_gp(gp_params(cur, nxt, fcap[nxt], (int64_t)hctr->bound_sum <= fcap[nxt]),
                                 tm.on ? &g1 : nullptr));
                cudaEvent_t g2 = tm.on ? tm.mark() : nullptr;
                if (tm.on) {
                    tm.span(T_GPW, g0, g1);
                    tm.span(T_GPB, g1, g2);
                }
                PLB_CK(cudaMemcpyAsync(hctr, ctr, sizeof(RoundCounters), cudaMemcpyDeviceToHost, s));
                PLB_CK(cudaStreamSynchronize(s));
                if (hctr->guard) return PLB_ERR_CUDA;
                if (!hctr->fovf) break;
                // new-frontier buffer too small: grow it and run the gather again
                const int64_t need = (int64_t)hctr->cursor;
                pool.release(fhub[nxt]);
                fcap[nxt] = need + need / 2 + 1024;
                fhub[nxt] = pool.alloc<uint32_t>(fcap[nxt]);
                PLB_ALLOC_OK();
                st.reruns += 1;
                rerun = true;
            }
        }
        const int64_t acc = (int64_t)hctr->accepted;
        if (d < PLB_MAX_ROUNDS) {
            // per distance d (summed over the batches of Alg. 4)
            st.receivers[d] += (int64_t)hctr->nR + hctr->nO1_base + hctr->nO2_base;
            st.accepted[d] += acc;
            st.unique_round[d] += (int64_t)hctr->uniq;
            st.prefiltered_round[d] += (int64_t)hctr->prefiltered;
            st.probed_round[d] += (int64_t)hctr->probed;
            st.messages_round[d] += (int64_t)hctr->msgs;
            host_stat[d] = 1;
            if (tm.on) round_ev.push_back({d, r0});
        }
        st.arcs_scanned += (int64_t)hctr->arcs;
        st.messages += (int64_t)hctr->msgs;
        st.unique_candidates += (int64_t)hctr->uniq;
        st.staged_entries += (int64_t)hctr->staged;
        st.probed_entries += (int64_t)hctr->probed;
        st.check_lv_entries += (int64_t)hctr->chk_lv;
        st.check_lh_entries += (int64_t)hctr->chk_lh;
        for (int k = 0; k < 3; ++k) st.tier_vertices[k] += (int64_t)hctr->tier[k];
        if (acc == 0) {
            finished = true;
            return PLB_OK;
        }
        if (d > PLB_MAX_DIST) {
            status = PLB_ERR_DIST_OVERFLOW;
            finished = true;
            return PLB_OK;
        }
        // merge: L <- L U dL_d (rows stay sorted by hub rank)
        cudaEvent_t m0 = tm.on ? tm.mark() : nullptr;
        const int64_t Tn = T + acc;
        if (Tn > lcap[nxt]) {
            pool.release(lent[nxt]);
            lcap[nxt] = Tn + Tn / 4 + 1024;
            lent[nxt] = pool.alloc<uint32_t>(lcap[nxt]);
            PLB_ALLOC_OK();
        }
        PLB_CK(launch_merge(cur, nxt));
        T = Tn;
        cur = nxt;
        if (d == 1 || acc > T - acc) {
            // most rows reach kIndexMinLen in round 1, and a round that more
            // than doubles the labels outgrows most tables: a packed rebuild
            // (cheaper than a new table per row from the shared pool cursor)
            const int e = build_index(cur, T, false);
            if (e != PLB_OK) return e;
        } else {
            PLB_CK(update_index(cur, T));  // a table that did not fit shows up as hovf at the next sync
        }
        if (tm.on) tm.span(T_MERGE, m0, tm.mark());
        // round-start reset of the per-round counters (nA carries over)
        PLB_CK(cudaMemsetAsync(ctr, 0, offsetof(RoundCounters, nA), s));
        PLB_CK(cudaMemsetAsync(&ctr->nO1_base, 0, sizeof(int) * 3, s));
        // grow the frontier buffer ahead of a large round
        if (acc > fcap[cur ^ 1] / 2) {
            const int nx2 = cur ^ 1;
            pool.release(fhub[nx2]);
            fcap[nx2] = 2 * acc + 1024;
            fhub[nx2] = pool.alloc<uint32_t>(fcap[nx2]);
            PLB_ALLOC_OK();
        }
        return PLB_OK;
    };

    // ---- graph mode: the round loop as one CUDA graph with a device-side while
    // condition (two rounds per body: the buffer parities alternate).  The graph
    // stops at a round that may not fit its buffers: before the gather when the
    // round's candidate bound exceeds the new-frontier buffer (the round then
    // continues host-driven), after it when its labels exceed the label buffers
    // (they grow and the round's merge runs here).  The graph is then captured
    // again and resumes with the next round.
    int rounds_total = 0;
    for (batch_lo = 0; batch_lo < n && status == PLB_OK; batch_lo += batch) {
        batch_hi = std::min<int64_t>(n, batch_lo + batch);
        if (batch_lo > 0) {
            // the previous batch ended with an empty round: restart the round count
            // and the per-round counters; its labels stay (the batches of Alg. 4
            // only restrict which hubs propagate)
            d = 0;
            finished = false;
            PLB_CK(cudaMemsetAsync(ctr, 0, offsetof(RoundCounters, nA), s));
            PLB_CK(cudaMemsetAsync(&ctr->nO1_base, 0, sizeof(int) * 3, s));
        }
        {  // round 1 is always host-driven (one kernel)
            const int e = host_round(false);
            if (e != PLB_OK) return e;
        }
        if (o.use_graph && batch == n && !finished) {
            RoundStat* dstat = pool.alloc<RoundStat>(PLB_MAX_ROUNDS);
            PLB_ALLOC_OK();
            PLB_CK(cudaMemsetAsync(dstat, 0, sizeof(RoundStat) * PLB_MAX_ROUNDS, s));
            int64_t lc = std::max<int64_t>(std::max<int64_t>(32 * n, T + 1024), 1 << 20);
            auto grow = [&](uint32_t*& buf, int64_t& cap, int64_t want, int64_t keep) -> bool {
                if (cap >= want) return true;
                uint32_t* nb = pool.alloc<uint32_t>(want);
                if (pool.failed) return false;
                if (keep > 0 &&
                    cudaMemcpyAsync(nb, buf, sizeof(uint32_t) * keep, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                    return false;
                pool.release(buf);
                buf = nb;
                cap = want;
                return true;
            };
            for (int attempt = 0; attempt < 8 && !finished; ++attempt) {
                if (!grow(lent[cur], lcap[cur], lc, T) || !grow(lent[cur ^ 1], lcap[cur ^ 1], lc, 0))
                    return PLB_ERR_OOM;
                {
                    const int e = build_index(cur, T, true);  // packed, with room for the segment's updates
                    if (e != PLB_OK) return e;
                }
                PLB_CK(cudaStreamSynchronize(s));
                hctr->d = (unsigned)d;
                hctr->cur = cur;
                hctr->T = T;
                hctr->lcap = std::min(lcap[0], lcap[1]);
                hctr->hcap = hcap;
                hctr->fcap[0] = fcap[0];
                hctr->fcap[1] = fcap[1];
                PLB_CK(cudaMemcpyAsync(&ctr->d, &hctr->d, sizeof(unsigned), cudaMemcpyHostToDevice, s));
                PLB_CK(cudaMemcpyAsync(&ctr->cur, &hctr->cur, sizeof(int), cudaMemcpyHostToDevice, s));
                PLB_CK(cudaMemcpyAsync(&ctr->T, &hctr->T, 5 * sizeof(long long), cudaMemcpyHostToDevice, s));
                cudaEvent_t ga = tm.on ? tm.mark() : nullptr;
                cudaGraph_t graph = nullptr;
                cudaGraphExec_t exec = nullptr;
                struct GraphGuard {
                    cudaGraph_t* g;
                    cudaGraphExec_t* e;
                    ~GraphGuard() {
                        if (*e) cudaGraphExecDestroy(*e);
                        if (*g) cudaGraphDestroy(*g);
                    }
                } gguard{&graph, &exec};
                PLB_CK(cudaGraphCreate(&graph, 0));
                cudaGraphConditionalHandle handle;
                PLB_CK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
                cudaGraphNodeParams cp = {};
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = handle;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                cudaGraphNode_t cnode;
                PLB_CK(cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp));
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                // capture on a private stream (capture is not allowed on the legacy
                // default stream); the graph itself is launched on the caller's stream
                cudaStream_t user_stream = s, cap_stream = nullptr;
                PLB_CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
                struct StreamGuard {
                    cudaStream_t st;
                    ~StreamGuard() { cudaStreamDestroy(st); }
                } sguard{cap_stream};
                s = cap_stream;
                skip = &ctr->done;
                PLB_CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
                cudaError_t ce = cudaSuccess;
                const int64_t launches0 = st.launches;
                for (int r = 0; r < 2 && ce == cudaSuccess; ++r) {
                    const int c = cur ^ r, x = c ^ 1;
                    k_g_begin<<<1, 1, 0, s>>>(ctr);
                    ce = launch_frontier(c, x);
                    if (ce == cudaSuccess) {
                        k_g_bound<<<1, 1, 0, s>>>(ctr, x);
                        ce = launch_gp(gp_params(c, x, fcap[x], true), nullptr);  // k_g_bound checked the bound
                    }
                    if (ce == cudaSuccess) {
                        k_g_check<<<1, 1, 0, s>>>(ctr, dstat);
                        ce = launch_merge(c, x);
                    }
                    if (ce == cudaSuccess) ce = update_index(x, T);
                    if (ce == cudaSuccess) {
                        k_g_finish<<<1, 1, 0, s>>>(ctr);
                        st.launches += 4;  // loop control
                        ce = cudaGetLastError();
                    }
                }
                k_g_cond<<<1, 1, 0, s>>>(ctr, handle);
                const cudaError_t ee = cudaStreamEndCapture(s, &body);
                s = user_stream;
                skip = nullptr;
                if (ce != cudaSuccess || ee != cudaSuccess) {
                    (void)cudaGetLastError();
                    set_last_error(ce != cudaSuccess ? ce : ee, __LINE__);
                    return PLB_ERR_CUDA;
                }
                const int64_t per_pair = st.launches - launches0 + 1;
                st.launches = launches0;
                PLB_CK(cudaGraphInstantiate(&exec, graph, 0));
                PLB_CK(cudaGraphLaunch(exec, s));
                PLB_CK(cudaMemcpyAsync(hctr, ctr, sizeof(RoundCounters), cudaMemcpyDeviceToHost, s));
                PLB_CK(cudaStreamSynchronize(s));
                if (tm.on) tm.span(T_GPW, ga, tm.mark());
                if (hctr->guard) return PLB_ERR_CUDA;
                const int dd = (int)hctr->d;  // last round started
                st.launches += per_pair * ((dd - d + 1) / 2);
                T = hctr->T;
                cur = hctr->cur;
                if (hctr->err) {
                    d = dd;
                    status = hctr->err;
                    finished = true;
                    break;
                }
                if (!hctr->fallback) {
                    d = dd;
                    finished = true;
                    break;
                }
                st.reruns += 1;
                PLB_CK(cudaMemsetAsync(&ctr->done, 0, sizeof(int) * 2, s));
                if (hctr->fallback == kStopIndex) {
                    // round dd is complete (parity flipped, counters reset); its probe
                    // index update did not fit: the next segment starts with a rebuild
                    d = dd;
                    continue;
                }
                if (hctr->fallback == kStopBeforeGather) {
                    // round dd's candidate bound exceeds the new-frontier buffer:
                    // the round continues host-driven from its gather
                    d = dd - 1;
                    const int e = host_round(true);
                    if (e != PLB_OK) return e;
                    continue;
                }
                if (hctr->fovf) {
                    // the new frontier of round dd overflowed its buffer: restore the
                    // round's start state and redo it host-driven
                    d = dd - 1;
                    hctr->nA = hctr->nA_saved;
                    PLB_CK(cudaMemsetAsync(ctr, 0, offsetof(RoundCounters, nA), s));
                    PLB_CK(cudaMemsetAsync(&ctr->nO1_base, 0, sizeof(int) * 3, s));
                    PLB_CK(cudaMemcpyAsync(&ctr->nA, &hctr->nA, sizeof(int), cudaMemcpyHostToDevice, s));
                    const int e = host_round(false);
                    if (e != PLB_OK) return e;
                    continue;
                }
                // the labels of round dd do not fit the label buffers: its gather is
                // complete, so grow the merge target and finish the round here
                const int nxt = cur ^ 1;
                const int64_t Tn = T + (int64_t)hctr->accepted;
                lc = std::max<int64_t>(Tn + Tn / 2, lc + lc / 2);
                if (!grow(lent[nxt], lcap[nxt], lc, 0)) return PLB_ERR_OOM;
                PLB_CK(launch_merge(cur, nxt));
                T = Tn;
                cur = nxt;
                d = dd;
                {
                    const int e = build_index(cur, T, true);
                    if (e != PLB_OK) return e;
                }
                PLB_CK(cudaMemsetAsync(ctr, 0, offsetof(RoundCounters, nA), s));
                PLB_CK(cudaMemsetAsync(&ctr->nO1_base, 0, sizeof(int) * 3, s));
            }
            // per-round statistics written on the device
            std::vector<RoundStat> hstat(PLB_MAX_ROUNDS);
            PLB_CK(cudaMemcpyAsync(hstat.data(), dstat, sizeof(RoundStat) * PLB_MAX_ROUNDS, cudaMemcpyDeviceToHost, s));
            PLB_CK(cudaStreamSynchronize(s));
            for (int r = 1; r <= d && r < PLB_MAX_ROUNDS; ++r) {
                if (host_stat[r]) continue;
                const RoundStat& x = hstat[r];
                st.receivers[r] = x.receivers;
                st.accepted[r] = x.accepted;
                st.unique_round[r] = x.uniq;
                st.prefiltered_round[r] = x.pref;
                st.probed_round[r] = x.probed;
                st.messages_round[r] = x.msgs;
                st.arcs_scanned += x.arcs;
                st.messages += x.msgs;
                st.unique_candidates += x.uniq;
                st.staged_entries += x.staged;
                st.probed_entries += x.probed;
                st.check_lv_entries += x.chk_lv;
                st.check_lh_entries += x.chk_lh;
                st.tier_vertices[0] += x.tier0;
                st.tier_vertices[1] += x.tier1;
            }
            // (after 8 graph segments the remaining rounds run host-driven)
        }

        // ---- host-driven rounds (from round d + 1)
        while (!finished) {
            const int e = host_round(false);
            if (e != PLB_OK) return e;
        }
        rounds_total += d;
    }  // batches
    st.rounds = rounds_total;
    st.total_labels = T;
    if (status != PLB_OK) return status;

    // ------------------------------------------------------------ finalize
    // only the final rows (loff, lent), the rank inverse, the scan buffers and
    // the counters are read from here on: the round buffers (probe index,
    // frontiers, tier scratch, masks, rank-space CSR) go back to the pool
    // before the label set is allocated, which lowers the build's peak
    pool.release_all_except({loff[cur], lent[cur], inv, tmp64, scan_scr, ctr});
    cudaEvent_t f0 = tm.on ? tm.mark() : nullptr;
    plb_labels* L = new plb_labels();
    L->n = n;
    L->total = T;
    L->rounds = st.rounds;
    auto fail = [&](int code) {
        if (L->off) cudaFreeAsync(L->off, s);
        if (L->packed) cudaFreeAsync(L->packed, s);
        if (L->hub) cudaFreeAsync(L->hub, s);
        if (L->dist) cudaFreeAsync(L->dist, s);
        if (L->order) cudaFreeAsync(L->order, s);
        delete L;
        return code;
    };
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
    if (cudaMemcpyAsync(L->order, order, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(PLB_ERR_CUDA);
    if (cudaMemcpyAsync(hctr, ctr, sizeof(RoundCounters), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return fail(PLB_ERR_CUDA);
    st.launches += 2 + scan_n;
    cudaEvent_t f1 = tm.on ? tm.mark() : nullptr;
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(PLB_ERR_CUDA);
    L->max_dist = (int32_t)hctr->max_dist;
    if (tm.on) {
        tm.span(T_FINAL, f0, f1);
        tm.span(T_ALL, t_all0, f1);
        st.ms_prepare = tm.total(T_PREP);
        st.ms_frontier = tm.total(T_FRONT);
        st.ms_gather_prune[0] = tm.total(T_GPW);
        st.ms_gather_prune[1] = tm.total(T_GPB);
        st.ms_gather_prune[2] = tm.total(T_GPG);
        st.ms_merge = tm.total(T_MERGE);
        st.ms_finalize = tm.total(T_FINAL);
        st.ms_total = tm.total(T_ALL);
        for (size_t i = 0; i < round_ev.size(); ++i) {
            cudaEvent_t end = i + 1 < round_ev.size() ? round_ev[i + 1].second : f0;
            float ms = 0;
            cudaEventElapsedTime(&ms, round_ev[i].second, end);
            st.ms_round[round_ev[i].first] += ms;
        }
    }
    L->stats = st;
    *out = L;
    return PLB_OK;
#undef PLB_CK
#undef PLB_ALLOC_OK
}

}  // namespace plb
