/*
 * plb.h -- C ABI of the GB300 (sm_103a) canonical 2-hop distance labeling
 * library ("pruned landmark labeling" built round by round, vertex-centric).
 *
 * Method: Jin, Peng, Wu, Dragan, Agrawal, Ren, "Pruned Landmark Labeling
 * Meets Vertex Centric Computation" (arXiv 1906.12018).
 *   - labels: Def. 2 (canonical hierarchical hub labeling, Sec. 2.1): for a
 *     total order pi, h is a hub of v iff h has the highest rank on every
 *     shortest h-v path; the label entry stores d(h, v).
 *   - construction: Alg. 3 (VC-PLL, Sec. 3.1), one vertex-centric round per
 *     distance d = 1, 2, ...; Thm. 1 shows it yields the labels of Def. 2.
 *   - query: Sec. 2.1, Dis(u,v) = min over common hubs h of d(u,h)+d(h,v).
 *   - variants (Sec. 5.1): directed graphs (plb_build_directed: L_in and
 *     L_out in the same rounds) and weighted graphs (plb_build_weighted:
 *     rounds by distance value); rank batches of Alg. 4 (plb_options.
 *     batch_hubs); many graphs in one round loop (plb_build_batch).
 *
 * General conventions
 *   - Every pointer argument that names graph, order, pair or distance data
 *     is a DEVICE pointer (CUDA global memory of the current device) unless
 *     its comment says "host".  Inputs are read-only for the duration of the
 *     call and stay owned by the caller.
 *   - Calls are ordered on the given stream (NULL = the legacy default
 *     stream).  The builds synchronise the stream internally (one or two
 *     device->host reads per round); plb_query_batch and
 *     plb_degree_order are asynchronous: results are ready when the stream is.
 *   - Vertices are int32 ids 0..n-1.  "rank" r in 0..n-1 is the position in
 *     the vertex order (rank 0 = highest); order[r] = id of rank r.
 *   - Limits: n < 2^24 (16,777,216 vertices; a label entry packs a 24-bit hub
 *     rank with an 8-bit distance), label distances <= 254.
 *   - Every entry point returns an int status (PLB_OK = 0) and never throws.
 *     On an error, no output object is created and nothing is returned
 *     through out-parameters.
 */
#ifndef PLB_H
#define PLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* plb_stream; /* == cudaStream_t */

/* ---------------------------------------------------------------- status */
enum plb_status {
    PLB_OK = 0,
    PLB_ERR_INVALID = 1,        /* bad argument, bad CSR, order not a permutation */
    PLB_ERR_OOM = 2,            /* device allocation failed */
    PLB_ERR_DIST_OVERFLOW = 3,  /* a label distance would exceed 254 */
    PLB_ERR_TIMEOUT = 4,        /* reserved for a bounded device-side wait that expired: no
                                 * kernel of this library waits on another (graph-mode round
                                 * loops end by the round limit), so no call returns it now */
    PLB_ERR_CUDA = 5,           /* a CUDA runtime call or launch failed */
    PLB_ERR_TOO_LARGE = 6       /* n >= 2^24 (or a weighted build's frontier ring too large) */
};

#define PLB_MAX_VERTICES (1 << 24)
#define PLB_MAX_DIST 254
#define PLB_UNREACHABLE (-1) /* query answer: s and t are in different components */
#define PLB_BAD_PAIR (-2)    /* query answer: s or t outside [0, n) */

/* Undirected unweighted graph as a symmetric CSR (device memory).
 * row_ptr[n+1] (row_ptr[0] = 0, row_ptr[n] = nnz, non-decreasing);
 * col[nnz] neighbour ids, each row strictly ascending (no duplicates), no
 * self-loops, and (u,v) present iff (v,u) present.  nnz = 2 * edges. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col;
} plb_csr;

/* Build options; plb_default_options fills the defaults. */
typedef struct {
    int32_t validate;          /* 1: check CSR and order on the device first (default 1) */
    int32_t warp_label_cap;    /* largest |L(v)| handled one-vertex-per-warp (default 512) */
    int32_t warp_cand_cap;     /* largest unique-candidate count per warp-vertex (default 512) */
    int32_t block_label_cap;   /* largest |L(v)| the block tier stages in shared memory (default 512) */
    int32_t block_cand_cap;    /* unique candidates per hub-range pass of the block tier (default 2048) */
    int32_t block_threads;     /* threads of the block tier, 64..256, rounded down to a multiple of 32 (default 256) */
    int32_t use_graph;         /* 1: run the rounds after round 1 as a captured CUDA graph with
                                  a device-side while condition (no per-round host sync);
                                  buffers get fixed capacities; a round that may not fit
                                  stops the graph, finishes host-driven after the buffers
                                  grow, and the graph resumes.  Ignored with batch_hubs.
                                  Default 0 (plb_build_batch without options: 1) */
    int32_t profile;           /* 1: time each kernel class with CUDA events */
    int32_t batch_hubs;        /* > 0: label in batches of this many hubs by rank (BVC-PLL,
                                  Alg. 4): the rounds of batch i propagate only the hubs of
                                  ranks [i*batch_hubs, (i+1)*batch_hubs); same labels.
                                  Default 0 (one batch: VC-PLL, Alg. 3) */
    int32_t warp_stage_ratio;  /* warp tier: a receiver whose candidate bound times this is below
                                  |L(v)| (a row with a probe table) looks L(v) up in v's row of
                                  the probe index instead of staging it in shared memory;
                                  0: always stage.  0..1024 (default 4) */
    int32_t reserved[6];
} plb_options;

/* Opaque label set (library-owned device memory; free with plb_labels_free). */
typedef struct plb_labels plb_labels;

/* Borrowed view of a label set: valid until plb_labels_free.
 * Rows indexed by ORIGINAL vertex id; entries of a row sorted by hub rank
 * ascending; hub = rank of the hub vertex; dist = d(hub, v) (0 for v itself). */
typedef struct {
    int64_t n;
    int64_t total;            /* sum of |L(v)| */
    const int64_t* off;       /* device, n+1 */
    const uint32_t* hub;      /* device, total */
    const uint8_t* dist;      /* device, total */
    const int32_t* order;     /* device, n: rank -> id used by the build */
    int32_t max_dist;         /* largest stored distance */
    int32_t rounds;           /* vertex-centric rounds executed (the last accepts nothing) */
} plb_label_view;

/* Counters and timings of one build (Sec. 3.3 / 4.3 cost terms). */
#define PLB_MAX_ROUNDS 256
typedef struct {
    int32_t rounds;
    int32_t reruns;                 /* gathers repeated after growing a buffer, and graph-mode stops */
    int64_t n, nnz, total_labels;
    /* per round d (index d, 1..rounds) */
    int64_t receivers[PLB_MAX_ROUNDS];   /* vertices that gathered messages */
    int64_t accepted[PLB_MAX_ROUNDS];    /* new labels (|dL_d|) */
    int64_t unique_round[PLB_MAX_ROUNDS];  /* distinct candidates checked in round d */
    int64_t probed_round[PLB_MAX_ROUNDS];  /* label entries probed in distance checks in round d */
    int64_t prefiltered_round[PLB_MAX_ROUNDS]; /* candidates pruned by the top-hub witness prefilter */
    int64_t messages_round[PLB_MAX_ROUNDS];/* frontier hubs h < v read by the gather in round d */
    double ms_round[PLB_MAX_ROUNDS];       /* device ms of round d (profile = 1 only) */
    /* totals over rounds */
    int64_t arcs_scanned;           /* neighbour entries read in the gather */
    int64_t messages;               /* frontier hubs h < v read by the gathers (before dedup) */
    int64_t unique_candidates;      /* distinct (h, v) pairs checked */
    int64_t staged_entries;         /* L(v) entries staged into the hub map */
    int64_t probed_entries;         /* L(h) or L(v) entries probed in distance checks */
    int64_t tier_vertices[3];       /* vertex-rounds: [0] round 1 and the warp tier, [1] block tier, [2] 0 */
    /* milliseconds on the device (profile = 1 only; else 0) */
    /* ms_gather_prune: [0] round 1 and the warp tier, [1] block tier (host-driven rounds run the two
       tiers concurrently: [1] is then the time the block tier outlasts the warp tier plus the
       escalated vertices), [2] 0 */
    double ms_total, ms_prepare, ms_frontier, ms_gather_prune[3], ms_merge, ms_finalize;
    int64_t launches;               /* kernels launched by this build */
    /* profile = 1 only (else 0): over the candidates (h, d) checked at v, the label entries the
       distance check reads by the cost model of Sec. 4.3: the entries of L(v) with hub < h (the
       side the paper scans), and |L(h)| (the side it hashes) */
    int64_t check_lv_entries;
    int64_t check_lh_entries;
} plb_build_stats;

/* Fill *opt with defaults. */
void plb_default_options(plb_options* opt);

/* Build the canonical labels (Def. 2) of g under vertex_order (device,
 * int32[n], rank -> id, a permutation of [0,n)) by vertex-centric rounds
 * (Alg. 3).  On success *out receives a new label set.
 * Errors: PLB_ERR_INVALID (null pointers, n < 0, nnz < 0, a CSR or order that
 * breaks the rules above -- checked on the device when opt->validate),
 * PLB_ERR_TOO_LARGE, PLB_ERR_OOM, PLB_ERR_DIST_OVERFLOW, PLB_ERR_CUDA. */
int plb_build(const plb_csr* g, const int32_t* vertex_order, const plb_options* opt,
              plb_stream stream, plb_labels** out);

/* Build k independent graphs in ONE round loop over their disjoint union
 * (host arrays gs[k], orders[k] of device pointers; outs[k] host array that
 * receives k label sets).  By Def. 2 a disjoint union's canonical labels,
 * under any order that keeps each part's own order, are the parts' labels,
 * so each outs[i] equals plb_build(&gs[i], orders[i]).  Parts are taken in
 * consecutive groups whose union has fewer than 2^24 vertices (one round loop
 * per group; each part itself must have fewer).  Errors as plb_build; on
 * error no label set is returned. */
int plb_build_batch(const plb_csr* gs, const int32_t* const* orders, int64_t k,
                    const plb_options* opt, plb_stream stream, plb_labels** outs);

/* Directed graphs (Sec. 5.1): g holds the OUT-arcs (row u lists the w with
 * an arc u -> w: strictly ascending, in range, no self-loops; the reverse arc
 * is NOT required).  Builds, in the same vertex-centric rounds, the
 * canonical in-labels (*l_in: row v holds (h, d(h -> v)) for the hubs h that
 * outrank every vertex of every shortest h -> v path) and out-labels
 * (*l_out: (h, d(v -> h)), likewise), each a label set as from plb_build.
 * Options as plb_build; use_graph and batch_hubs are ignored (host-driven
 * rounds, one batch).  Errors as plb_build; on error neither set is returned. */
int plb_build_directed(const plb_csr* g, const int32_t* vertex_order, const plb_options* opt,
                       plb_stream stream, plb_labels** l_in, plb_labels** l_out);

/* Weighted graphs (Sec. 5.1): g as for plb_build (symmetric CSR, device);
 * weight (device, uint8[nnz]) is the weight of arc j (the arc to col[j]),
 * at least 1 and equal in both directions.  Builds the canonical labels of
 * Def. 2 over weighted shortest paths: (h, d(h,v)) is in L(v) iff h outranks
 * every vertex of every shortest h-v path; the label set has the layout of
 * plb_build's (distances are weighted, at most PLB_MAX_DIST) and is queried
 * with plb_query_batch.  Rounds follow the distance: round d accepts the
 * labels at distance d from the candidates that the frontiers of rounds
 * d - w send over arcs of weight w, checked against the labels of distance
 * below d (the snapshot test of Alg. 3), so the result is canonical without
 * the end-of-batch recheck of Sec. 5.1.  Device memory grows with the
 * largest weight (one frontier descriptor per vertex and round of the last
 * max-weight rounds).  Options as plb_build; use_graph and batch_hubs are
 * ignored (host-driven rounds, one batch).  Errors as plb_build, and
 * PLB_ERR_INVALID for a null weight array with arcs or a zero weight (always
 * checked) or, with validate, a weight that differs from its reverse arc's;
 * PLB_ERR_TOO_LARGE when (largest weight + 1) * 2^ceil(log2 n) + 1 >= 2^31. */
int plb_build_weighted(const plb_csr* g, const uint8_t* weight, const int32_t* vertex_order,
                       const plb_options* opt, plb_stream stream, plb_labels** out);

/* Answer q distance queries (Sec. 2.1): pairs (device, int32[2q],
 * s_i = pairs[2i], t_i = pairs[2i+1], original ids) -> dist_out (device,
 * int32[q]): d(s,t), PLB_UNREACHABLE if no common hub, PLB_BAD_PAIR if an id
 * is outside [0,n).  Asynchronous on the stream; returns PLB_ERR_INVALID for
 * null pointers or q < 0. */
int plb_query_batch(const plb_labels* labels, const int32_t* pairs, int64_t q,
                    int32_t* dist_out, plb_stream stream);

/* Directed queries: dist_out[i] = d(s_i -> t_i) = min over hubs h of
 * l_out(s_i) and l_in(t_i) of d(s_i -> h) + d(h -> t_i), from the two sets of
 * one plb_build_directed; codes as plb_query_batch.  PLB_ERR_INVALID when
 * the sets have different vertex counts. */
int plb_query_directed(const plb_labels* l_out, const plb_labels* l_in, const int32_t* pairs, int64_t q,
                       int32_t* dist_out, plb_stream stream);

/* Same query over several label sets in one launch: pair i is answered on
 * sets[set_idx[i]] (set_idx device int32[q]); sets is a host array of m label
 * sets that must all stay alive until the stream reaches this work.  A pair
 * whose set index is outside [0,m) gets PLB_BAD_PAIR. */
int plb_query_multi(const plb_labels* const* sets, int64_t m, const int32_t* set_idx,
                    const int32_t* pairs, int64_t q, int32_t* dist_out, plb_stream stream);

/* Borrow device pointers of a label set. */
int plb_labels_view(const plb_labels* labels, plb_label_view* view);

/* Counters/timings of the build that produced the label set. */
int plb_labels_stats(const plb_labels* labels, plb_build_stats* stats);

/* Device bytes held by a label set. */
int64_t plb_labels_bytes(const plb_labels* labels);

/* Release a label set (synchronises the device first). NULL is accepted. */
int plb_labels_free(plb_labels* labels);

/* The library allocates from its own stream-ordered pool per device and keeps
 * freed blocks for reuse by later builds.  This returns every cached,
 * currently unused block to the driver (synchronises the device). */
int plb_release_cached_memory(void);

/* Device memory of the library's pool on the current device, in bytes:
 * out[0] in use now, out[1] the most in use at once since the last reset,
 * out[2] reserved from the driver now, out[3] the most reserved at once.
 * out: host int64[4] (caller-owned).  reset != 0 then restarts both high
 * marks from the current values (a build's peak is out[1] read after it
 * with a reset before it).  Returns PLB_ERR_INVALID for a NULL out,
 * PLB_ERR_CUDA when the pool cannot be queried; all zeros before the
 * library's first allocation on the device. */
int plb_memory_stats(int64_t* out, int reset);

/* Degree order (Sec. 6.1: vertices ordered by degree): order_out (device,
 * int32[n]) receives rank -> id, degree descending, ties by smaller id.
 * Only row_ptr is read.  Allocates device scratch (8 bytes per vertex,
 * rounded up to a power of two).  Asynchronous on the stream. */
int plb_degree_order(const plb_csr* g, int32_t* order_out, plb_stream stream);

/* Allocation-free degree order (no counterpart in the paper; a service of
 * this library).  Same result as plb_degree_order, for callers that cannot
 * let the library allocate device memory: processes whose device memory is
 * owned by a host framework's allocator, servers that admit work against a
 * fixed HBM budget, and latency-critical paths where cudaMalloc/cudaFree may
 * block or synchronise the device.  It calls no allocating routine: its
 * scratch is a fixed array of PLB_NOALLOC_MAX_VERTICES 8-byte keys (8 MiB)
 * inside the library, held on every GPU that loads the library until the
 * process exits.
 *   - n > PLB_NOALLOC_MAX_VERTICES -> PLB_ERR_TOO_LARGE, nothing launched.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device.
 *   - All calls share the one array (each call rewrites the part it uses
 *     before reading it): calls whose work overlaps on the GPU -- on
 *     different streams, or from several host threads -- race and must be
 *     serialised by the caller.
 *   - Otherwise as plb_degree_order: row_ptr read, order_out (device,
 *     int32[n]) written, asynchronous on the stream. */
#define PLB_NOALLOC_MAX_VERTICES (1 << 20)
int plb_degree_order_noalloc(const plb_csr* g, int32_t* order_out, plb_stream stream);

/* Human-readable status text (static storage). */
const char* plb_strerror(int status);

/* Where the last PLB_ERR_CUDA of a build on this host thread came from: the
 * library call site and CUDA's error name and text (static, thread-local
 * storage; "" if none). */
const char* plb_last_error(void);

/* ABI version: 100 * major + minor. */
int plb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PLB_H */
