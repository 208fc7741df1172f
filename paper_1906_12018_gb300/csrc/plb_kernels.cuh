// Kernels of the vertex-centric labeling rounds (Alg. 3, Sec. 3.1), in rank
// space: vertex i is the vertex of rank i, so "h outranks v" is h < v.
//
// Round 1 is k_round1 (no candidate can be pruned).  Per round d >= 2
// (labels L and frontier dL_{d-1} as they stood after round d-1):
//   k_mark         every active a (dL_{d-1}(a) non-empty) flags the neighbours
//                  v that some hub of dL_{d-1}(a) outranks (scatter, Alg. 3).
//   k_collect      flagged vertices become this round's receivers, routed by
//                  their candidate bound, |L(v)| and degree to a tier.
//   k_gp_warp      gather + dedup + distance check, one vertex per warp, with
//                  L(v) staged hub-keyed in shared memory (the gather of
//                  Alg. 3: unique messages, then d < min over common hubs).
//   k_gp_block     the same with one vertex per block (any size: hub-range
//                  passes, a byte map for the top hubs).
//   k_sort_rows_*  rows of the new frontier that were written unsorted (round
//                  1; the block tier's) sorted by hub rank (the warp tier
//                  writes its rows sorted);
//   k_merge_*      L(v) <- L(v) U dL_d(v), keeping rows sorted by hub rank;
//                  then the probe index of L is rebuilt (k_index_*).
#pragma once

#include "plb_internal.cuh"

namespace plb {

struct RoundCounters {
    unsigned long long cursor;    // append cursor of the new frontier buffer
    unsigned long long accepted;  // new labels this round
    unsigned long long arcs, msgs, uniq, staged, probed;
    unsigned long long tier[3];
    unsigned long long bound_sum; // sum over receivers of the candidate bound min(v, messages)
    unsigned long long prefiltered; // candidates pruned by the top-hub witness prefilter
    unsigned long long chk_lv, chk_lh;  // checked candidates (h at v): sums of |L(v) entries with hub < h|
                                        // and of |L(h)| (counted when GpParams::count_check is set)
    int nR, nO1, nO2;             // receivers: warp tier, block tier (nO2 unused)
    int nBig, nGiant;             // new frontier rows too long for a warp / for shared memory to sort
    int nU;                       // vertices whose new frontier row was written unsorted (block tier)
    int nA;                       // next active list (kept across the per-round reset)
    int nO1_base, nO2_base;       // tier-list sizes made by k_collect (for reruns)
    int fovf;                     // new-frontier buffer overflow
    unsigned int max_dist;        // finalize: largest stored distance
    int guard;                    // a kernel met a broken capacity invariant (internal error)
    // loop control (kept across rounds)
    unsigned int d;               // current round (distance of the labels being accepted)
    int done;                     // no further round runs; round kernels return at once
    int fallback;                 // graph mode stopped at a capacity limit: resume on the host
    int err;                      // status set by the device (PLB_ERR_DIST_OVERFLOW)
    int nA_saved;                 // active count of the current round (restored on fallback)
    int cur;                      // buffer parity holding L and the previous frontier
    long long T;                  // labels so far (graph mode)
    long long lcap, hcap;         // label and probe-index buffer capacities (graph mode)
    long long fcap[2];            // new-frontier buffer capacity per parity (graph mode)
    long long hnext;              // probe index: first free table slot
    int hovf;                     // probe index: a table did not fit (the index must be rebuilt)
};

// RoundCounters::fallback: why a graph stopped (1: after the gather, a buffer
// was too small; kStopBeforeGather: the candidate bound exceeds the frontier
// buffer; kStopIndex: after a complete round, the probe index needs a rebuild).
constexpr int kStopBeforeGather = 2;
constexpr int kStopIndex = 3;

// Per-round statistics written on the device (graph mode).
struct RoundStat {
    long long receivers, accepted, uniq, probed, msgs, pref, arcs, staged, tier0, tier1, chk_lv, chk_lh;
};

struct GpParams {
    const int64_t* roff;
    const int32_t* rcol;
    const int64_t* loff;
    const uint32_t* lent;
    const uint64_t* fse;       // frontier of round d-1: start|count per vertex
    const uint32_t* fhub;      // frontier hubs of round d-1 (rows sorted)
    uint64_t* fse_new;         // frontier of round d
    uint32_t* fhub_new;
    unsigned long long fcap;   // capacity of fhub_new
    const int32_t* list;       // vertices handled by this tier
    const int* list_n;
    int32_t* esc;              // escalation list (next tier)
    int* esc_n;
    RoundCounters* ctr;        // also holds the round number d (ctr->d)
    int log_s, log_m;          // table sizes (log2 slots): candidate set, L(v) map (block tier: largest)
    int cand_limit;            // max unique candidates per pass (power of two)
    uint32_t* gscratch;        // block tier: per-block buffer of accepted hubs
    int64_t gscratch_words;    // words per block
    const uint64_t* hdesc;     // probe index of L: per row (table start << 8 | log2 slots), 0 = no table
    const uint32_t* htab;
    const uint32_t* top;       // per vertex: top-hub masks by distance level (see kTopHubs)
    // The candidates' side of the check: rows, probe index and top-hub masks
    // of the labels h contributes (the same arrays as above for undirected
    // graphs; for L_in(v) of a directed graph the L_out of h, and vice versa).
    const int64_t* loff_h;
    const uint32_t* lent_h;
    const uint64_t* hdesc_h;
    const uint32_t* htab_h;
    const uint32_t* top_h;
    const uint4* hrec_h;       // per vertex of the candidates' side, or null: {row start << 24 | row length
                               // (64 bits), probe-table descriptor (64 bits)}, one 16-byte load per check
    const uint32_t* rbound;    // per receiver: candidate bound min(v, messages)
    const int64_t* ostart;     // per receiver: start of its new frontier row (the scan of the bounds),
                               // or null (rows reserved with an atomic cursor)
    int stage_ratio;           // warp tier: L(v) read from v's probe table when rbound[v] * stage_ratio
                               // < |L(v)| (0: always staged in shared memory)
    int32_t* unsorted;         // block tier: list of the vertices whose new row it wrote (unsorted;
                               // count ctr->nU), or null (every new row is sorted after the round)
    int sender_bits;           // rcol holds frontier descriptor indices whose low sender_bits bits are
                               // the sending vertex (weighted rounds), or 0: the vertex itself
    int count_check;           // 1: count the label entries each check would read by the paper's cost
                               // model (RoundCounters::chk_lv / chk_lh; one binary search per candidate)
};

// The sending vertex of an arc's descriptor index (see GpParams::sender_bits).
__device__ __forceinline__ uint32_t sender_of(const GpParams& p, int32_t a) {
    return p.sender_bits ? (uint32_t)a & ((1u << p.sender_bits) - 1u) : (uint32_t)a;
}

// Witness prefilter: for the kTopHubs highest-ranked hubs, every vertex x
// keeps kTopLevels bitmasks C_t(x) = {w : w in L(x), d(w, x) <= t}, t = 1..
// kTopLevels (8 words each).  A candidate h at round d has a witness among
// those hubs when E_i(v) & C_{d-i}(h) != 0 for some i, E_i = C_i & ~C_{i-1}:
// the label test restricted to those hubs and distances (exact: a hit is a
// real witness).
#ifndef PLB_TOP_HUBS
#define PLB_TOP_HUBS 256
#endif
constexpr int kTopHubs = PLB_TOP_HUBS;  // a multiple of 128 (uint4 loads)
static_assert(kTopHubs % 128 == 0, "top-hub masks are read as uint4");
constexpr int kTopWords = kTopHubs / 32;             // words per mask
constexpr int kTopLevels = 7;                        // distance levels 1..7
constexpr int kTopRow = kTopLevels * kTopWords;      // words per vertex

// Messages each lane loads before inserting them (gathers keep several loads
// in flight per warp).
constexpr int kGatherUnroll = 4;
// Label entries each lane loads per step of a distance check.
constexpr int kCheckUnroll = 2;

// Block tier: hubs below this rank are deduplicated in a shared-memory byte
// map (one byte per hub) instead of the hash set.
constexpr int kByteHubs = 32768;
// Receivers whose candidate bound reaches this use the byte map (for fewer
// candidates clearing and scanning it costs more than the hashing it saves).
constexpr uint32_t kByteMinBound = 2048;
constexpr int kByteStage = 160;  // per-warp staging of byte-map candidates (< 32 carried + 128 new)

// Rows of L with at least this many entries get a hub-keyed probe table.
constexpr int kIndexMinLen = 16;
// k_index_build: warps per block, and the largest table a warp may build in
// its shared-memory buffer (larger ones are filled in place).  The buffer is
// chosen per launch: 512 slots (16 KB per block, eight blocks per SM) while
// the rows are short, 2048 when they are long.
constexpr int kIndexWarps = 8;
constexpr int kIndexSmemSlotsMax = 2048;

// Check records (GpParams::hrec_h): row start << 24 | length, then the
// probe-table descriptor (table start << 8 | log2 slots, below 2^48) with the
// row's count of entries whose hub is below kTopHubs in its top 16 bits.
__host__ __device__ __forceinline__ uint64_t hrec_row(uint64_t start, uint64_t len) { return (start << 24) | len; }
constexpr int kHrecTopShift = 16;  // within the record's last word
constexpr uint64_t kHrecDescMask = (uint64_t(1) << 48) - 1;
__global__ void k_pack_hrec(const int64_t* loff, const uint32_t* lent, const uint64_t* hdesc, uint4* hrec, int64_t n,
                            const RoundCounters* ctr);

// Routing limits of k_collect (see the tier geometry in build_core).
struct TierLimits {
    int64_t warp_bound;   // candidate bound up to which the warp tier is tried
    int64_t warp_label;   // largest |L(v)| of the warp tier
    int64_t warp_deg;     // largest degree of the warp tier
};

struct WarpSync {
    __device__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
    __device__ void operator()() const { __syncthreads(); }
};

}  // namespace plb
