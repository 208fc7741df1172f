// Host driver of the directed labeling (Sec. 5.1): L_in(v) holds (h, d(h->v))
// and L_out(v) holds (h, d(v->h)) for the hubs h that outrank every vertex of
// every shortest path between them.  Both are built in the same rounds:
// round d propagates dL_in along out-arcs (v gathers the new L_in hubs of its
// in-neighbours) and dL_out along in-arcs (v gathers from its out-neighbours);
// a candidate (h, d) for L_in(v) is pruned by a hub w with
// d(h->w) + d(w->v) <= d read from L_out(h) and L_in(v), one for L_out(v) by
// d(v->w) + d(w->h) from L_out(v) and L_in(h); both sides read the labels of
// round d - 1 and merge after both gathers.  The kernels are those of the
// undirected build with the candidate's side of the check pointed at the
// other direction's labels.  Host-driven rounds only (no graph mode, one
// batch).
#include <algorithm>
#include <cstring>
#include <vector>

#include "plb_host.cuh"

namespace plb {

namespace {

// One direction: its labels, frontier, probe index, masks, lists, counters.
struct Side {
    const int64_t* g_off = nullptr;  // gather arcs: the neighbours whose new hubs v reads
    const int32_t* g_col = nullptr;
    const int64_t* s_off = nullptr;  // scatter arcs: the vertices an active a sends to
    const int32_t* s_col = nullptr;
    int64_t* loff[2] = {nullptr, nullptr};
    uint32_t* lent[2] = {nullptr, nullptr};
    int64_t lcap[2] = {0, 0};
    uint64_t* fse[2] = {nullptr, nullptr};
    uint32_t* fhub[2] = {nullptr, nullptr};
    int64_t fcap[2] = {0, 0};
    uint32_t* top = nullptr;
    int64_t* hoff = nullptr;
    uint64_t* hdesc = nullptr;
    uint32_t* htab = nullptr;
    int64_t hcap = 0;
    unsigned long long* recv = nullptr;
    int32_t* A = nullptr;
    int32_t* R = nullptr;
    int32_t* O1 = nullptr;
    int32_t* U = nullptr;           // vertices whose new row the block tier wrote unsorted
    uint32_t* rbound = nullptr;
    int64_t* aoff = nullptr;
    RoundCounters* ctr = nullptr;
    RoundCounters* hctr = nullptr;  // pinned host mirror
    int cur = 0;                    // parity of the current labels and frontier
    int64_t T = 0;                  // labels so far
    bool done = false;              // no new labels in the last round: none will follow
    int rounds = 0;
    plb_build_stats st{};
};

}  // namespace

int build_directed_core(const int64_t* row_ptr, const int32_t* col, const int32_t* order, int64_t n, int64_t nnz,
                        const plb_options& o, cudaStream_t s, plb_labels** out_in, plb_labels** out_out) {
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
    cudaEvent_t t_all0 = tm.on ? tm.mark() : nullptr;
    int64_t launches = 0;

    Side side[2];  // 0: L_in, 1: L_out
    int* err = pool.alloc<int>(4);
    for (int k = 0; k < 2; ++k) side[k].ctr = pool.alloc<RoundCounters>(1);
    PLB_ALLOC_OK();
    RoundCounters* hbuf = nullptr;
    PLB_CK(cudaMallocHost(&hbuf, 2 * sizeof(RoundCounters)));
    struct HostFree {
        void* p;
        ~HostFree() { cudaFreeHost(p); }
    } hf{hbuf};
    for (int k = 0; k < 2; ++k) {
        side[k].hctr = hbuf + k;
        PLB_CK(cudaMemsetAsync(side[k].ctr, 0, sizeof(RoundCounters), s));
    }
    PLB_CK(cudaMemsetAsync(err, 0, 4 * sizeof(int), s));

    cudaEvent_t t0 = tm.on ? tm.mark() : nullptr;
    // ---------------------------------------------------------- validation
    if (o.validate) {
        k_check_rowptr<<<grid_for(n + 1, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(row_ptr, n, nnz, err);
        int* seen = pool.alloc<int>(n);
        PLB_ALLOC_OK();
        PLB_CK(cudaMemsetAsync(seen, 0, sizeof(int) * std::max<int64_t>(n, 1), s));
        int herr = 0;
        PLB_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PLB_CK(cudaStreamSynchronize(s));
        if (herr) return PLB_ERR_INVALID;
        if (nnz > 0)
            k_check_cols<<<grid_for((nnz + 2047) / 2048, 1, flat_grid_cap), kFlatThreads, 0, s>>>(row_ptr, col, n,
                                                                                               nnz, 0, err);
        k_check_order<<<grid_for(n, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(order, n, seen, err);
        PLB_CK(cudaGetLastError());
        PLB_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PLB_CK(cudaStreamSynchronize(s));
        launches += 3;
        pool.release(seen);
        if (herr) return PLB_ERR_INVALID;
    }

    // ------------------------------------- rank-space arcs and their transpose
    int32_t* inv = pool.alloc<int32_t>(n);
    int64_t* roff_o = pool.alloc<int64_t>(n + 1);
    int32_t* rcol_o = pool.alloc<int32_t>(nnz);
    int64_t* roff_i = pool.alloc<int64_t>(n + 1);
    int32_t* rcol_i = pool.alloc<int32_t>(nnz);
    int64_t* tmp64 = pool.alloc<int64_t>(n + 1);
    int64_t* scan_scr = pool.alloc<int64_t>(scan_scratch_elems(n + 1));
    PLB_ALLOC_OK();
    const int scan_n = scan_launch_count(n);
    k_inverse<<<gflat, kFlatThreads, 0, s>>>(order, inv, n);
    k_rank_degree<<<gflat, kFlatThreads, 0, s>>>(row_ptr, order, tmp64, n);
    PLB_CK(cudaGetLastError());
    PLB_CK(exclusive_scan_i64(tmp64, roff_o, n, scan_scr, s));
    PLB_CK(cudaMemsetAsync(tmp64, 0, sizeof(int64_t) * (n + 1), s));
    if (nnz > 0) {
        k_relabel<<<grid_for((nnz + 2047) / 2048, 1, flat_grid_cap), kFlatThreads, 0, s>>>(row_ptr, col, order, inv,
                                                                                          roff_o, rcol_o, n, nnz);
        k_in_degree<<<grid_for(nnz, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(rcol_o, nnz, tmp64);
    }
    PLB_CK(exclusive_scan_i64(tmp64, roff_i, n, scan_scr, s));
    if (nnz > 0) {
        unsigned long long* fill = reinterpret_cast<unsigned long long*>(tmp64);
        PLB_CK(cudaMemsetAsync(fill, 0, sizeof(unsigned long long) * n, s));
        k_transpose<<<grid_for((nnz + 2047) / 2048, 1, flat_grid_cap), kFlatThreads, 0, s>>>(roff_o, rcol_o, n, nnz,
                                                                                            roff_i, fill, rcol_i);
    }
    PLB_CK(cudaGetLastError());
    launches += 6 + 2 * scan_n;
    // L_in(v) gathers from v's in-neighbours, whose new hubs travel along
    // their out-arcs; L_out the other way round
    side[0].g_off = roff_i;
    side[0].g_col = rcol_i;
    side[0].s_off = roff_o;
    side[0].s_col = rcol_o;
    side[1].g_off = roff_o;
    side[1].g_col = rcol_o;
    side[1].s_off = roff_i;
    side[1].s_col = rcol_i;

    // ------------------------------------------------------------ state
    for (int k = 0; k < 2; ++k) {
        Side& S = side[k];
        for (int b = 0; b < 2; ++b) {
            S.lcap[b] = std::max<int64_t>(2 * n, 1024);
            S.loff[b] = pool.alloc<int64_t>(n + 1);
            S.lent[b] = pool.alloc<uint32_t>(S.lcap[b]);
            S.fcap[b] = std::max<int64_t>(nnz + n, 1024);  // round 1 adds at most one label per arc
            S.fse[b] = pool.alloc<uint64_t>(n);
            S.fhub[b] = pool.alloc<uint32_t>(S.fcap[b]);
        }
        S.top = pool.alloc<uint32_t>(n * kTopRow);
        S.hoff = pool.alloc<int64_t>(n + 1);
        S.hdesc = pool.alloc<uint64_t>(n);
        S.hcap = std::max<int64_t>(4 * n, 1024);
        S.htab = pool.alloc<uint32_t>(S.hcap);
        S.recv = pool.alloc<unsigned long long>(n);
        S.A = pool.alloc<int32_t>(n);
        S.R = pool.alloc<int32_t>(n);
        S.O1 = pool.alloc<int32_t>(n);
        S.U = pool.alloc<int32_t>(n);
        S.rbound = pool.alloc<uint32_t>(n);
        S.aoff = pool.alloc<int64_t>(n + 1);
        PLB_ALLOC_OK();
        PLB_CK(cudaMemsetAsync(S.recv, 0, sizeof(unsigned long long) * std::max<int64_t>(n, 1), s));
        k_init<<<gflat, kFlatThreads, 0, s>>>(S.s_off, n, S.loff[0], S.lent[0], S.fse[0], S.fhub[0], S.A, S.ctr);
        k_top_init<<<flat_grid_cap, kFlatThreads, 0, s>>>(S.top, n);
        PLB_CK(cudaGetLastError());
        S.T = n;
        S.st.n = n;
        S.st.nnz = nnz;
        launches += 2;
    }
    PLB_CK(cudaFuncSetAttribute(k_index_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(uint32_t) * kIndexWarps * kIndexSmemSlotsMax)));
    PLB_CK(cudaFuncSetAttribute(k_index_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(uint32_t) * kIndexWarps * kIndexSmemSlotsMax)));
    auto index_slots = [&](int64_t total) { return total <= 128 * n ? 512 : kIndexSmemSlotsMax; };
    // packed rebuild of side k's probe index (room for growth)
    auto build_index = [&](Side& S) -> int {
        const int64_t total = S.T;
        if (S.hcap < 6 * total + 1024) {
            pool.release(S.htab);
            S.hcap = 8 * total + 1024;
            S.htab = pool.alloc<uint32_t>(S.hcap);
            if (pool.failed) return PLB_ERR_OOM;
        }
        k_index_size<<<gflat, kFlatThreads, 0, s>>>(S.loff[S.cur], n, tmp64, S.ctr);
        if (exclusive_scan_i64(tmp64, S.hoff, n, scan_scr, s) != cudaSuccess) return PLB_ERR_CUDA;
        const int slots = index_slots(total);
        k_index_build<<<grid_for((n + 255) / 256, 1, flat_grid_cap), kIndexWarps * 32,
                        sizeof(uint32_t) * kIndexWarps * slots, s>>>(S.loff[S.cur], S.lent[S.cur], S.hoff, S.htab,
                                                                     S.hdesc, n, slots, S.ctr);
        k_index_total<<<1, 1, 0, s>>>(S.hoff, n, S.ctr);
        launches += 3 + scan_n;
        return cudaGetLastError() == cudaSuccess ? PLB_OK : PLB_ERR_CUDA;
    };
    for (int k = 0; k < 2; ++k) {
        const int e = build_index(side[k]);
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
    PLB_CK(cudaFuncSetAttribute(k_sort_rows_radix, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortRadixSmemBytes));
    int occ_w = 1, occ_b = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_w, k_gp_warp, kGpWarpThreads, w_smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, k_gp_block, bthr, b_smem);
    const int grid_w = sms * std::max(1, occ_w);
    const int grid_b = sms * std::max(1, occ_b);
    int32_t* big = pool.alloc<int32_t>(n);
    int32_t* giant = pool.alloc<int32_t>(n);
    uint32_t* cur1 = pool.alloc<uint32_t>(n);  // round 1: per-row write cursors
    const int sort_blocks = 8;
    const int64_t sort_words = pow2_at_least(std::max<int64_t>(n, 1));
    uint32_t* sortscr = pool.alloc<uint32_t>(sort_words * sort_blocks);
    uint32_t* gacc = pool.alloc<uint32_t>((int64_t)grid_b * std::max<int64_t>(n, 1));
    PLB_ALLOC_OK();

    // ------------------------------------------------------------ rounds
    auto frontier = [&](Side& S) -> cudaError_t {
        const int c = S.cur, x = c ^ 1;
        k_active_degree<<<gflat, kFlatThreads, 0, s>>>(S.s_off, S.A, S.ctr, tmp64, n);
        cudaError_t e = exclusive_scan_i64(tmp64, S.aoff, n, scan_scr, s);
        if (e != cudaSuccess) return e;
        k_mark<<<flat_grid_cap, kFlatThreads, 0, s>>>(S.s_off, S.s_col, S.fse[c], S.fhub[c], S.A, S.aoff, S.ctr,
                                                      S.recv, n);
        k_collect<<<gflat, kFlatThreads, 0, s>>>(S.recv, S.g_off, S.loff[c], n, S.fse[x], S.R, S.O1, S.rbound, nullptr,
                                                 S.ctr, lim);
        k_after_collect<<<1, 1, 0, s>>>(S.ctr);
        launches += 4 + scan_n;
        return cudaGetLastError();
    };
    // gather + prune of side S; the candidates' side of the check is side H
    auto gather = [&](Side& S, const Side& H) -> cudaError_t {
        const int c = S.cur, x = c ^ 1;
        GpParams p{};
        p.roff = S.g_off;
        p.rcol = S.g_col;
        p.loff = S.loff[c];
        p.lent = S.lent[c];
        p.fse = S.fse[c];
        p.fhub = S.fhub[c];
        p.fse_new = S.fse[x];
        p.fhub_new = S.fhub[x];
        p.fcap = (unsigned long long)S.fcap[x];
        p.ctr = S.ctr;
        p.hdesc = S.hdesc;
        p.htab = S.htab;
        p.top = S.top;
        p.loff_h = H.loff[H.cur];
        p.lent_h = H.lent[H.cur];
        p.hdesc_h = H.hdesc;
        p.htab_h = H.htab;
        p.top_h = H.top;
        p.gscratch = gacc;
        p.gscratch_words = std::max<int64_t>(n, 1);
        p.rbound = S.rbound;
        p.list = S.R;
        p.list_n = &S.ctr->nR;
        p.esc = S.O1;
        p.esc_n = &S.ctr->nO1;
        p.log_s = w_log_s;
        p.log_m = w_log_m;
        p.cand_limit = warp_cand;
        p.stage_ratio = o.warp_stage_ratio;
        p.count_check = o.profile != 0;
        p.unsorted = S.U;
        k_gp_warp<<<grid_w, kGpWarpThreads, w_smem, s>>>(p);
        p.list = S.O1;
        p.list_n = &S.ctr->nO1;
        p.esc = nullptr;
        p.esc_n = nullptr;
        p.log_s = b_log_s;
        p.log_m = b_log_m;
        p.cand_limit = block_cand;
        k_gp_block<<<grid_b, bthr, b_smem, s>>>(p);
        launches += 2;
        return cudaGetLastError();
    };
    auto merge = [&](Side& S) -> cudaError_t {
        const int c = S.cur, x = c ^ 1;
        k_next_active<<<gflat, kFlatThreads, 0, s>>>(S.loff[c], S.fse[x], n, tmp64, S.A, S.ctr);
        k_sort_rows_warp<<<sms * 8, 256, 0, s>>>(S.fse[x], S.fhub[x], S.A, S.U, 1, S.ctr, big, giant);
        k_sort_rows_radix<<<sms, 1024, kSortRadixSmemBytes, s>>>(S.fse[x], S.fhub[x], big, &S.ctr->nBig, S.ctr);
        k_sort_rows_block<<<sort_blocks, 1024, 16384 * sizeof(uint32_t), s>>>(S.fse[x], S.fhub[x], giant,
                                                                            &S.ctr->nGiant, sortscr, sort_words,
                                                                            S.ctr);
        cudaError_t e = exclusive_scan_i64(tmp64, S.loff[x], n, scan_scr, s);
        if (e != cudaSuccess) return e;
        k_merge_old<<<flat_grid_cap, kFlatThreads, 0, s>>>(S.loff[c], S.lent[c], S.loff[x], S.lent[x], S.fse[x],
                                                           S.fhub[x], n, S.ctr);
        k_merge_new<<<grid_for((int64_t)n * 32, kFlatThreads, flat_grid_cap), kFlatThreads, 0, s>>>(
            S.loff[c], S.lent[c], S.loff[x], S.lent[x], S.fse[x], S.fhub[x], S.A, S.ctr, S.top);
        launches += 6 + scan_n;
        return cudaGetLastError();
    };
    auto read_ctr = [&](Side& S) -> cudaError_t {
        return cudaMemcpyAsync(S.hctr, S.ctr, sizeof(RoundCounters), cudaMemcpyDeviceToHost, s);
    };

    int status = PLB_OK;
    int d = 0;
    while (!(side[0].done && side[1].done)) {
        ++d;
        cudaEvent_t r0 = tm.on ? tm.mark() : nullptr;
        // gather both sides on the labels of round d - 1
        for (int k = 0; k < 2; ++k) {
            Side& S = side[k];
            if (S.done) continue;
            const int x = S.cur ^ 1;
            k_set_round<<<1, 1, 0, s>>>(S.ctr, (uint32_t)d);
            launches += 1;
            if (d == 1) {
                const int g1 = grid_for((nnz + 2047) / 2048, 1, flat_grid_cap);
                PLB_CK(cudaMemsetAsync(tmp64, 0, sizeof(int64_t) * (n + 1), s));
                PLB_CK(cudaMemsetAsync(cur1, 0, sizeof(uint32_t) * std::max<int64_t>(n, 1), s));
                if (nnz > 0)
                    k_round1_count<<<g1, kFlatThreads, 0, s>>>(S.g_off, S.g_col, n, nnz, 0, (int32_t)n,
                                                              reinterpret_cast<unsigned long long*>(tmp64), S.ctr);
                PLB_CK(exclusive_scan_i64(tmp64, tmp64, n, scan_scr, s));
                k_round1<<<g1, kFlatThreads, 0, s>>>(S.g_off, S.g_col, n, nnz, 0, (int32_t)n, tmp64, cur1, S.fse[x],
                                                    S.fhub[x], (unsigned long long)S.fcap[x], S.ctr);
                launches += 2 + scan_n;
                PLB_CK(cudaGetLastError());
                continue;
            }
            PLB_CK(frontier(S));
        }
        for (int k = 0; k < 2 && d > 1; ++k) {
            Side& S = side[k];
            if (S.done) continue;
            const int x = S.cur ^ 1;
            PLB_CK(read_ctr(S));
            PLB_CK(cudaStreamSynchronize(s));
            if (S.hctr->hovf) {
                const int e = build_index(S);
                if (e != PLB_OK) return e;
            }
            if ((int64_t)S.hctr->bound_sum > S.fcap[x]) {
                const int64_t want = std::min<int64_t>((int64_t)S.hctr->bound_sum + 1024,
                                                       std::max<int64_t>(int64_t(1) << 31, 2 * S.fcap[x]));
                if (want > S.fcap[x]) {
                    pool.release(S.fhub[x]);
                    S.fcap[x] = want;
                    S.fhub[x] = pool.alloc<uint32_t>(S.fcap[x]);
                    PLB_ALLOC_OK();
                }
            }
        }
        if (tm.on) tm.span(T_FRONT, r0, tm.mark());
        cudaEvent_t g0 = tm.on ? tm.mark() : nullptr;
        for (int k = 0; k < 2 && d > 1; ++k) {
            Side& S = side[k];
            if (S.done) continue;
            for (int attempt = 0;; ++attempt) {
                if (attempt > 0) {
                    k_rerun_reset<<<gflat, kFlatThreads, 0, s>>>(S.ctr, S.fse[S.cur ^ 1], n);
                    launches += 1;
                }
                PLB_CK(gather(S, side[k ^ 1]));
                PLB_CK(read_ctr(S));
                PLB_CK(cudaStreamSynchronize(s));
                if (S.hctr->guard) return PLB_ERR_CUDA;
                if (!S.hctr->fovf) break;
                const int x = S.cur ^ 1;  // new-frontier buffer too small: grow it, gather again
                const int64_t need = (int64_t)S.hctr->cursor;
                pool.release(S.fhub[x]);
                S.fcap[x] = need + need / 2 + 1024;
                S.fhub[x] = pool.alloc<uint32_t>(S.fcap[x]);
                PLB_ALLOC_OK();
                S.st.reruns += 1;
            }
        }
        for (int k = 0; k < 2 && d == 1; ++k) {
            PLB_CK(read_ctr(side[k]));
            PLB_CK(cudaStreamSynchronize(s));
            if (side[k].hctr->fovf) return PLB_ERR_CUDA;  // cannot happen: the buffer holds every arc
        }
        if (tm.on) tm.span(T_GPW, g0, tm.mark());
        // statistics; a side that accepted nothing is finished
        for (int k = 0; k < 2; ++k) {
            Side& S = side[k];
            if (S.done) continue;
            const RoundCounters& h = *S.hctr;
            const int64_t acc = (int64_t)h.accepted;
            if (d < PLB_MAX_ROUNDS) {
                S.st.receivers[d] = (int64_t)h.nR + h.nO1_base + h.nO2_base;
                S.st.accepted[d] = acc;
                S.st.unique_round[d] = (int64_t)h.uniq;
                S.st.prefiltered_round[d] = (int64_t)h.prefiltered;
                S.st.probed_round[d] = (int64_t)h.probed;
                S.st.messages_round[d] = (int64_t)h.msgs;
            }
            S.st.arcs_scanned += (int64_t)h.arcs;
            S.st.messages += (int64_t)h.msgs;
            S.st.unique_candidates += (int64_t)h.uniq;
            S.st.staged_entries += (int64_t)h.staged;
            S.st.probed_entries += (int64_t)h.probed;
            S.st.check_lv_entries += (int64_t)h.chk_lv;
            S.st.check_lh_entries += (int64_t)h.chk_lh;
            for (int q = 0; q < 3; ++q) S.st.tier_vertices[q] += (int64_t)h.tier[q];
            S.rounds = d;
            if (acc == 0) S.done = true;
            else if (d > PLB_MAX_DIST) status = PLB_ERR_DIST_OVERFLOW;
        }
        if (status != PLB_OK) break;
        // merges after both gathers (snapshot of round d - 1 for both checks)
        cudaEvent_t m0 = tm.on ? tm.mark() : nullptr;
        for (int k = 0; k < 2; ++k) {
            Side& S = side[k];
            if (S.done) continue;
            const int x = S.cur ^ 1;
            const int64_t Tn = S.T + (int64_t)S.hctr->accepted;
            if (Tn > S.lcap[x]) {
                pool.release(S.lent[x]);
                S.lcap[x] = Tn + Tn / 4 + 1024;
                S.lent[x] = pool.alloc<uint32_t>(S.lcap[x]);
                PLB_ALLOC_OK();
            }
            PLB_CK(merge(S));
            const int64_t Told = S.T;
            S.T = Tn;
            S.cur = x;
            if (d == 1 || Tn - Told > Told) {  // round 1, or a round that more than doubles the labels: repack
                const int e = build_index(S);
                if (e != PLB_OK) return e;
            } else {
                const int slots = index_slots(S.T);
                k_index_update<<<flat_grid_cap, kIndexWarps * 32, sizeof(uint32_t) * kIndexWarps * slots, s>>>(
                    S.loff[x], S.lent[x], S.fse[x], S.fhub[x], S.A, S.htab, S.hdesc, (long long)S.hcap, slots,
                    S.ctr);
                launches += 1;
                PLB_CK(cudaGetLastError());
            }
            PLB_CK(cudaMemsetAsync(S.ctr, 0, offsetof(RoundCounters, nA), s));
            PLB_CK(cudaMemsetAsync(&S.ctr->nO1_base, 0, sizeof(int) * 3, s));
            if ((int64_t)S.hctr->accepted > S.fcap[S.cur ^ 1] / 2) {  // grow the next frontier buffer ahead
                const int nx2 = S.cur ^ 1;
                pool.release(S.fhub[nx2]);
                S.fcap[nx2] = 2 * (int64_t)S.hctr->accepted + 1024;
                S.fhub[nx2] = pool.alloc<uint32_t>(S.fcap[nx2]);
                PLB_ALLOC_OK();
            }
        }
        if (tm.on) tm.span(T_MERGE, m0, tm.mark());
    }
    if (status != PLB_OK) return status;

    // ------------------------------------------------------------ finalize
    // the round buffers go back to the pool before the label sets are allocated
    pool.release_all_except({side[0].loff[side[0].cur], side[0].lent[side[0].cur], side[1].loff[side[1].cur],
                             side[1].lent[side[1].cur], side[0].ctr, side[1].ctr, inv, tmp64, scan_scr});
    cudaEvent_t f0 = tm.on ? tm.mark() : nullptr;
    plb_labels* Lk[2] = {nullptr, nullptr};
    auto fail = [&](int code) {
        for (plb_labels* L : Lk) {
            if (!L) continue;
            if (L->off) cudaFreeAsync(L->off, s);
            if (L->packed) cudaFreeAsync(L->packed, s);
            if (L->hub) cudaFreeAsync(L->hub, s);
            if (L->dist) cudaFreeAsync(L->dist, s);
            if (L->order) cudaFreeAsync(L->order, s);
            delete L;
        }
        return code;
    };
    for (int k = 0; k < 2; ++k) {
        Side& S = side[k];
        const int64_t T = S.T;
        plb_labels* L = Lk[k] = new plb_labels();
        L->n = n;
        L->total = T;
        L->rounds = S.rounds;
        if (plb::dev_alloc((void**)&L->off, sizeof(int64_t) * (n + 1), s) != cudaSuccess ||
            plb::dev_alloc((void**)&L->packed, sizeof(uint32_t) * std::max<int64_t>(T, 1), s) != cudaSuccess ||
            plb::dev_alloc((void**)&L->hub, sizeof(uint32_t) * std::max<int64_t>(T, 1), s) != cudaSuccess ||
            plb::dev_alloc((void**)&L->dist, std::max<int64_t>(T, 1), s) != cudaSuccess ||
            plb::dev_alloc((void**)&L->order, sizeof(int32_t) * std::max<int64_t>(n, 1), s) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(PLB_ERR_OOM);
        }
        L->bytes = (int64_t)(sizeof(int64_t) * (n + 1) + 9 * (size_t)T + 4 * (size_t)n);
        k_final_len<<<gflat, kFlatThreads, 0, s>>>(S.loff[S.cur], inv, n, tmp64);
        if (exclusive_scan_i64(tmp64, L->off, n, scan_scr, s) != cudaSuccess) return fail(PLB_ERR_CUDA);
        k_finalize<<<grid_for((T + 2047) / 2048, 1, flat_grid_cap), kFlatThreads, 0, s>>>(
            S.loff[S.cur], S.lent[S.cur], inv, L->off, L->packed, L->hub, L->dist, n, S.ctr);
        if (cudaMemcpyAsync(L->order, order, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            read_ctr(S) != cudaSuccess)
            return fail(PLB_ERR_CUDA);
        launches += 2 + scan_n;
    }
    cudaEvent_t f1 = tm.on ? tm.mark() : nullptr;
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(PLB_ERR_CUDA);
    for (int k = 0; k < 2; ++k) {
        Side& S = side[k];
        Lk[k]->max_dist = (int32_t)S.hctr->max_dist;
        S.st.rounds = S.rounds;
        S.st.total_labels = S.T;
        S.st.launches = launches;
        if (tm.on) {
            if (k == 0) {
                tm.span(T_FINAL, f0, f1);
                tm.span(T_ALL, t_all0, f1);
            }
            S.st.ms_prepare = tm.total(T_PREP);
            S.st.ms_frontier = tm.total(T_FRONT);
            S.st.ms_gather_prune[0] = tm.total(T_GPW);  // both sides
            S.st.ms_merge = tm.total(T_MERGE);
            S.st.ms_finalize = tm.total(T_FINAL);
            S.st.ms_total = tm.total(T_ALL);
        }
        Lk[k]->stats = S.st;
    }
    *out_in = Lk[0];
    *out_out = Lk[1];
    return PLB_OK;
#undef PLB_CK
#undef PLB_ALLOC_OK
}

}  // namespace plb
