// Exported C entry points: options, single and batched builds, label views.
#include <algorithm>
#include <atomic>
#include <vector>

#include "plb_internal.cuh"

namespace plb {

int build_core(const int64_t* row_ptr, const int32_t* col, const int32_t* order, int64_t n, int64_t nnz,
               const plb_options& o, cudaStream_t s, plb_labels** out, int64_t max_part_n);
int build_directed_core(const int64_t* row_ptr, const int32_t* col, const int32_t* order, int64_t n, int64_t nnz,
                        const plb_options& o, cudaStream_t s, plb_labels** out_in, plb_labels** out_out);
int build_weighted_core(const int64_t* row_ptr, const int32_t* col, const uint8_t* wt, const int32_t* order,
                        int64_t n, int64_t nnz, const plb_options& o, cudaStream_t s, plb_labels** out);
extern thread_local char g_last_error[256];

namespace {

// Storage shared by the label sets of one batched build.
struct Shared {
    std::atomic<int> refs{0};
    void* ptrs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

struct GraphDesc {
    const int64_t* row_ptr;
    const int32_t* col;
    const int32_t* order;
    int64_t vbase, ebase, n, nnz;
};

__device__ __forceinline__ int find_part(const int64_t* base, int k, int64_t x) {
    int lo = 0, hi = k - 1;  // largest g with base[g] <= x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Disjoint union: vertex u of part g becomes vbase[g] + u; the union order
// lists part 0's order, then part 1's, ... (each part keeps its own order).
__global__ void k_union_rows(const GraphDesc* gd, const int64_t* vb, int k, int64_t N, int64_t E, int64_t* U_off,
                             int32_t* U_ord) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < N; u += (int64_t)gridDim.x * blockDim.x) {
        const int g = find_part(vb, k, u);
        const GraphDesc d = gd[g];
        const int64_t lu = u - d.vbase;
        U_off[u] = d.ebase + d.row_ptr[lu];
        U_ord[u] = d.order[lu] + (int32_t)d.vbase;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) U_off[N] = E;
}

__global__ void k_union_cols(const GraphDesc* gd, const int64_t* eb, int k, int64_t E, int32_t* U_col) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int g = find_part(eb, k, e);
        const GraphDesc d = gd[g];
        U_col[e] = d.col[e - d.ebase] + (int32_t)d.vbase;
    }
}

// Split the union's labels into per-part rows: offsets rebased per part
// (part g's n_g+1 offsets start at vbase[g] + g), hubs shifted back.
__global__ void k_split_offsets(const int64_t* off, const int64_t* vb, int k, int64_t N, int64_t* off_all) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < N + k; u += (int64_t)gridDim.x * blockDim.x) {
        // position u of off_all belongs to part g where vb[g] + g <= u
        int lo = 0, hi = k - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (vb[mid] + mid <= u) lo = mid; else hi = mid - 1;
        }
        const int g = lo;
        const int64_t j = u - (vb[g] + g);  // 0..n_g
        off_all[u] = off[vb[g] + j] - off[vb[g]];
    }
}

__global__ void k_split_entries(const int64_t* eoff, int k, int64_t T, const int64_t* vb, uint32_t* packed,
                                uint32_t* hub, int32_t* order, int64_t N) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < T; q += (int64_t)gridDim.x * blockDim.x) {
        const int g = find_part(eoff, k, q);
        const uint32_t sh = (uint32_t)vb[g];
        const uint32_t e = packed[q];
        packed[q] = pack(hub_of(e) - sh, dist_of(e));
        hub[q] = hub_of(e) - sh;
    }
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < N; u += (int64_t)gridDim.x * blockDim.x) {
        const int g = find_part(vb, k, u);
        order[u] -= (int32_t)vb[g];
    }
}

__global__ void k_gather_eoff(const int64_t* off, const int64_t* vb, int k, int64_t* eoff) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= k; g += gridDim.x * blockDim.x) eoff[g] = off[vb[g]];
}

int grid_of(int64_t items) {
    int64_t b = (items + 255) / 256;
    if (b < 1) b = 1;
    if (b > 8192) b = 8192;
    return (int)b;
}

}  // namespace
}  // namespace plb

extern "C" {

void plb_default_options(plb_options* o) {
    if (!o) return;
    *o = plb_options{};
    o->validate = 1;
    o->warp_label_cap = 512;
    o->warp_cand_cap = 512;
    o->block_label_cap = 512;
    o->block_cand_cap = 2048;
    o->block_threads = 256;
    o->use_graph = 0;
    o->profile = 0;
    o->batch_hubs = 0;
    o->warp_stage_ratio = 4;
}

static int check_csr(const plb_csr* g, const int32_t* order) {
    if (!g || g->n < 0 || g->nnz < 0) return PLB_ERR_INVALID;
    if (g->n >= PLB_MAX_VERTICES) return PLB_ERR_TOO_LARGE;
    if (g->n > 0 && (!g->row_ptr || !order)) return PLB_ERR_INVALID;
    if (g->nnz > 0 && !g->col) return PLB_ERR_INVALID;
    if (g->n == 0 && g->nnz != 0) return PLB_ERR_INVALID;
    return PLB_OK;
}

static bool sane_options(const plb_options& o) {
    return o.warp_label_cap >= 1 && o.warp_label_cap <= 8192 && o.warp_cand_cap >= 1 && o.warp_cand_cap <= 4096 &&
           o.block_label_cap >= 1 && o.block_label_cap <= 16384 && o.block_cand_cap >= 1 &&
           o.block_cand_cap <= 16384 && o.block_threads >= 64 && o.block_threads <= 256 && o.batch_hubs >= 0 &&
           o.warp_stage_ratio >= 0 && o.warp_stage_ratio <= 1024;
}

static int empty_labels(plb_labels** out, cudaStream_t s) {
    plb_labels* L = new plb_labels();
    if (plb::dev_alloc((void**)&L->off, sizeof(int64_t), s) != cudaSuccess ||
        cudaMemsetAsync(L->off, 0, sizeof(int64_t), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        delete L;
        return PLB_ERR_CUDA;
    }
    *out = L;
    return PLB_OK;
}

int plb_build(const plb_csr* g, const int32_t* vertex_order, const plb_options* opt, plb_stream stream,
              plb_labels** out) {
    if (!out) return PLB_ERR_INVALID;
    const int c = check_csr(g, vertex_order);
    if (c != PLB_OK) return c;
    plb_options o;
    if (opt) o = *opt; else plb_default_options(&o);
    if (!sane_options(o)) return PLB_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    if (g->n == 0) return empty_labels(out, s);
    return plb::build_core(g->row_ptr, g->col, vertex_order, g->n, g->nnz, o, s, out, g->n);
}

int plb_build_directed(const plb_csr* g, const int32_t* vertex_order, const plb_options* opt, plb_stream stream,
                       plb_labels** l_in, plb_labels** l_out) {
    if (!l_in || !l_out) return PLB_ERR_INVALID;
    const int c = check_csr(g, vertex_order);
    if (c != PLB_OK) return c;
    plb_options o;
    if (opt) o = *opt; else plb_default_options(&o);
    if (!sane_options(o)) return PLB_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    if (g->n == 0) {
        const int e = empty_labels(l_in, s);
        if (e != PLB_OK) return e;
        const int e2 = empty_labels(l_out, s);
        if (e2 != PLB_OK) plb_labels_free(*l_in);
        return e2;
    }
    return plb::build_directed_core(g->row_ptr, g->col, vertex_order, g->n, g->nnz, o, s, l_in, l_out);
}

int plb_build_weighted(const plb_csr* g, const uint8_t* weight, const int32_t* vertex_order, const plb_options* opt,
                       plb_stream stream, plb_labels** out) {
    if (!out) return PLB_ERR_INVALID;
    const int c = check_csr(g, vertex_order);
    if (c != PLB_OK) return c;
    if (g->nnz > 0 && !weight) return PLB_ERR_INVALID;
    plb_options o;
    if (opt) o = *opt; else plb_default_options(&o);
    if (!sane_options(o)) return PLB_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    if (g->n == 0) return empty_labels(out, s);
    return plb::build_weighted_core(g->row_ptr, g->col, weight, vertex_order, g->n, g->nnz, o, s, out);
}

// One round loop over the disjoint union of parts [0, k) of gs/orders.
static int build_union(const plb_csr* gs, const int32_t* const* orders, int64_t k, const plb_options& o,
                       cudaStream_t s, plb_labels** outs) {
    std::vector<plb::GraphDesc> hd((size_t)k);
    std::vector<int64_t> vb((size_t)k + 1), eb((size_t)k + 1);
    int64_t N = 0, E = 0;
    for (int64_t i = 0; i < k; ++i) {
        vb[i] = N;
        eb[i] = E;
        hd[i] = {gs[i].row_ptr, gs[i].col, orders[i], N, E, gs[i].n, gs[i].nnz};
        N += gs[i].n;
        E += gs[i].nnz;
    }
    vb[k] = N;
    eb[k] = E;
    // device copies of the part table
    plb::GraphDesc* dgd = nullptr;
    int64_t *dvb = nullptr, *deb = nullptr, *U_off = nullptr, *eoff = nullptr;
    int32_t *U_col = nullptr, *U_ord = nullptr;
    auto cleanup = [&]() {
        for (void* p : {(void*)dgd, (void*)dvb, (void*)deb, (void*)U_off, (void*)eoff, (void*)U_col, (void*)U_ord})
            if (p) cudaFreeAsync(p, s);
    };
    if (plb::dev_alloc((void**)&dgd, sizeof(plb::GraphDesc) * k, s) != cudaSuccess ||
        plb::dev_alloc((void**)&dvb, sizeof(int64_t) * (k + 1), s) != cudaSuccess ||
        plb::dev_alloc((void**)&deb, sizeof(int64_t) * (k + 1), s) != cudaSuccess ||
        plb::dev_alloc((void**)&eoff, sizeof(int64_t) * (k + 1), s) != cudaSuccess ||
        plb::dev_alloc((void**)&U_off, sizeof(int64_t) * (N + 1), s) != cudaSuccess ||
        plb::dev_alloc((void**)&U_col, sizeof(int32_t) * std::max<int64_t>(E, 1), s) != cudaSuccess ||
        plb::dev_alloc((void**)&U_ord, sizeof(int32_t) * std::max<int64_t>(N, 1), s) != cudaSuccess) {
        (void)cudaGetLastError();
        cleanup();
        return PLB_ERR_OOM;
    }
    if (cudaMemcpyAsync(dgd, hd.data(), sizeof(plb::GraphDesc) * k, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dvb, vb.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(deb, eb.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cleanup();
        return PLB_ERR_CUDA;
    }
    if (N > 0) plb::k_union_rows<<<plb::grid_of(N), 256, 0, s>>>(dgd, dvb, (int)k, N, E, U_off, U_ord);
    if (E > 0) plb::k_union_cols<<<plb::grid_of(E), 256, 0, s>>>(dgd, deb, (int)k, E, U_col);
    if (cudaGetLastError() != cudaSuccess) {
        cleanup();
        return PLB_ERR_CUDA;
    }
    plb_labels* U = nullptr;
    int64_t max_part = 1;  // a vertex accepts hubs of its own graph only
    for (int64_t i = 0; i < k; ++i) max_part = std::max<int64_t>(max_part, gs[i].n);
    int st = N > 0 ? plb::build_core(U_off, U_col, U_ord, N, E, o, s, &U, max_part) : empty_labels(&U, s);
    if (st != PLB_OK) {
        cleanup();
        return st;
    }
    // split into per-part label sets sharing the union's storage
    int64_t* off_all = nullptr;
    if (plb::dev_alloc((void**)&off_all, sizeof(int64_t) * (N + k), s) != cudaSuccess) {
        (void)cudaGetLastError();
        cleanup();
        plb_labels_free(U);
        return PLB_ERR_OOM;
    }
    plb::k_split_offsets<<<plb::grid_of(N + k), 256, 0, s>>>(U->off, dvb, (int)k, N, off_all);
    plb::k_gather_eoff<<<1, 256, 0, s>>>(U->off, dvb, (int)k, eoff);
    if (U->total > 0 || N > 0)
        plb::k_split_entries<<<plb::grid_of(std::max<int64_t>(U->total, N)), 256, 0, s>>>(
            eoff, (int)k, U->total, dvb, U->packed, U->hub, U->order, N);
    std::vector<int64_t> heoff((size_t)k + 1);
    if (cudaMemcpyAsync(heoff.data(), eoff, sizeof(int64_t) * (k + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        cudaFreeAsync(off_all, s);
        cleanup();
        plb_labels_free(U);
        return PLB_ERR_CUDA;
    }
    auto* sh = new plb::Shared();
    sh->ptrs[0] = off_all;
    sh->ptrs[1] = U->packed;
    sh->ptrs[2] = U->hub;
    sh->ptrs[3] = U->dist;
    sh->ptrs[4] = U->order;
    sh->refs = (int)k;
    for (int64_t i = 0; i < k; ++i) {
        plb_labels* L = new plb_labels();
        L->n = gs[i].n;
        L->off = off_all + vb[i] + i;
        L->packed = U->packed + heoff[i];
        L->hub = U->hub + heoff[i];
        L->dist = U->dist + heoff[i];
        L->order = U->order + vb[i];
        L->total = heoff[i + 1] - heoff[i];
        L->max_dist = U->max_dist;
        L->rounds = U->rounds;
        L->stats = U->stats;
        L->bytes = (int64_t)(sizeof(int64_t) * (L->n + 1) + 9 * (size_t)L->total + 4 * (size_t)L->n);
        L->shared = sh;
        outs[i] = L;
    }
    // U's arrays now belong to the shared block; release only U->off
    cudaFreeAsync(U->off, s);
    delete U;
    cleanup();
    cudaStreamSynchronize(s);
    return PLB_OK;
}

int plb_build_batch(const plb_csr* gs, const int32_t* const* orders, int64_t k, const plb_options* opt,
                    plb_stream stream, plb_labels** outs) {
    if (k < 0 || (k > 0 && (!gs || !orders || !outs))) return PLB_ERR_INVALID;
    if (k == 0) return PLB_OK;
    if (k > (1 << 24)) return PLB_ERR_TOO_LARGE;
    plb_options o;
    if (opt) {
        o = *opt;
    } else {
        plb_default_options(&o);
        o.use_graph = 1;  // many small graphs: the round loop runs as one captured graph
    }
    if (!sane_options(o)) return PLB_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    for (int64_t i = 0; i < k; ++i) {
        const int c = check_csr(&gs[i], orders[i]);
        if (c != PLB_OK) return c;
    }
    // consecutive groups of parts whose union stays below 2^24 vertices; one
    // round loop per group
    int64_t lo = 0;
    while (lo < k) {
        int64_t hi = lo, nsum = 0;
        while (hi < k && nsum + gs[hi].n < PLB_MAX_VERTICES) nsum += gs[hi++].n;
        const int st = build_union(gs + lo, orders + lo, hi - lo, o, s, outs + lo);
        if (st != PLB_OK) {
            for (int64_t i = 0; i < lo; ++i) {
                plb_labels_free(outs[i]);
                outs[i] = nullptr;
            }
            return st;
        }
        lo = hi;
    }
    return PLB_OK;
}

int plb_labels_view(const plb_labels* L, plb_label_view* v) {
    if (!L || !v) return PLB_ERR_INVALID;
    v->n = L->n;
    v->total = L->total;
    v->off = L->off;
    v->hub = L->hub;
    v->dist = L->dist;
    v->order = L->order;
    v->max_dist = L->max_dist;
    v->rounds = L->rounds;
    return PLB_OK;
}

int plb_labels_stats(const plb_labels* L, plb_build_stats* st) {
    if (!L || !st) return PLB_ERR_INVALID;
    *st = L->stats;
    return PLB_OK;
}

int64_t plb_labels_bytes(const plb_labels* L) { return L ? L->bytes : 0; }

int plb_labels_free(plb_labels* L) {
    if (!L) return PLB_OK;
    (void)cudaGetLastError();  // report this call's failures (a sticky error shows again below)
    cudaDeviceSynchronize();
    if (L->shared) {
        auto* sh = static_cast<plb::Shared*>(L->shared);
        if (--sh->refs == 0) {
            for (void* p : sh->ptrs)
                if (p) cudaFreeAsync(p, 0);
            delete sh;
        }
    } else {
        for (void* p : {(void*)L->off, (void*)L->packed, (void*)L->hub, (void*)L->dist, (void*)L->order})
            if (p) cudaFreeAsync(p, 0);
    }
    delete L;
    // the blocks came from the library's stream-ordered pool: freed in stream
    // order they return to it for the next build (its use counts drop), and
    // the frees have completed when this returns
    cudaDeviceSynchronize();
    return cudaGetLastError() == cudaSuccess ? PLB_OK : PLB_ERR_CUDA;
}

const char* plb_strerror(int status) {
    switch (status) {
        case PLB_OK: return "ok";
        case PLB_ERR_INVALID: return "invalid argument, graph or order";
        case PLB_ERR_OOM: return "device out of memory";
        case PLB_ERR_DIST_OVERFLOW: return "label distance above 254";
        case PLB_ERR_TIMEOUT: return "device-side wait timed out";
        case PLB_ERR_CUDA: return "CUDA error";
        case PLB_ERR_TOO_LARGE: return "graph too large (n >= 2^24)";
        default: return "unknown status";
    }
}

int plb_version(void) { return 100; }

const char* plb_last_error(void) { return plb::g_last_error; }

}  // extern "C"
