// Declarations of the round kernels (plb_round.cu; the gather + prune kernels
// k_gp_warp and k_gp_block in plb_gather.cu).
#pragma once

#include "plb_kernels.cuh"

namespace plb {

__global__ void k_check_rowptr(const int64_t* row_ptr, int64_t n, int64_t nnz, int* err);
__global__ void k_check_cols(const int64_t* row_ptr, const int32_t* col, int64_t n, int64_t nnz, int symmetric,
                             int* err);
__global__ void k_in_degree(const int32_t* rcol, int64_t nnz, int64_t* indeg);
__global__ void k_transpose(const int64_t* roff, const int32_t* rcol, int64_t n, int64_t nnz, const int64_t* roff_t,
                            unsigned long long* fill, int32_t* rcol_t);
__global__ void k_check_order(const int32_t* order, int64_t n, int* seen, int* err);
__global__ void k_inverse(const int32_t* order, int32_t* inv, int64_t n);
__global__ void k_rank_degree(const int64_t* row_ptr, const int32_t* order, int64_t* rdeg, int64_t n);
__global__ void k_relabel(const int64_t* row_ptr, const int32_t* col, const int32_t* order, const int32_t* inv,
                          const int64_t* roff, int32_t* rcol, int64_t n, int64_t nnz);
__global__ void k_init(const int64_t* roff, int64_t n, int64_t* loff, uint32_t* lent, uint64_t* fse,
                       uint32_t* fhub, int32_t* A, RoundCounters* ctr);
__global__ void k_active_degree(const int64_t* roff, const int32_t* A, const RoundCounters* ctr, int64_t* adeg,
                                int64_t n);
__global__ void k_mark(const int64_t* roff, const int32_t* rcol, const uint64_t* fse, const uint32_t* fhub,
                       const int32_t* A, const int64_t* aoff, const RoundCounters* ctr, unsigned long long* recv,
                       int64_t n);
__global__ void k_collect(unsigned long long* recv, const int64_t* roff, const int64_t* loff, int64_t n,
                          uint64_t* fse_new, int32_t* R, int32_t* O1, uint32_t* rbound, int64_t* obound,
                          RoundCounters* ctr, TierLimits lim);
__global__ void k_after_collect(RoundCounters* ctr);
__global__ void k_rerun_reset(RoundCounters* ctr, uint64_t* fse_new, int64_t n);
__global__ void k_round1_count(const int64_t* roff, const int32_t* rcol, int64_t n, int64_t nnz, int32_t s,
                               int32_t e, unsigned long long* cnt, const RoundCounters* ctr);
__global__ void k_round1(const int64_t* roff, const int32_t* rcol, int64_t n, int64_t nnz, int32_t s, int32_t e,
                         const int64_t* start, uint32_t* cur, uint64_t* fse_new, uint32_t* fhub_new,
                         unsigned long long fcap, RoundCounters* ctr);
__global__ void k_gp_warp(GpParams p);
__global__ void k_gp_block(GpParams p);
__global__ void k_index_size(const int64_t* loff, int64_t n, int64_t* hsz, const RoundCounters* ctr);
__global__ void k_index_build(const int64_t* loff, const uint32_t* lent, const int64_t* hoff, uint32_t* htab,
                              uint64_t* hdesc, int64_t n, int slots, const RoundCounters* ctr);
__global__ void k_index_total(const int64_t* hoff, int64_t n, RoundCounters* ctr);
__global__ void k_index_update(const int64_t* loff, const uint32_t* lent, const uint64_t* fse_new,
                               const uint32_t* fhub_new, const int32_t* A, uint32_t* htab, uint64_t* hdesc,
                               long long hcap, int slots, RoundCounters* ctr);
__global__ void k_set_round(RoundCounters* ctr, uint32_t d);
__global__ void k_g_begin(RoundCounters* ctr);
__global__ void k_g_bound(RoundCounters* ctr, int x);
__global__ void k_g_check(RoundCounters* ctr, RoundStat* stats);
__global__ void k_g_finish(RoundCounters* ctr);
__global__ void k_g_cond(const RoundCounters* ctr, cudaGraphConditionalHandle h);
__global__ void k_next_active(const int64_t* loff, const uint64_t* fse_new, int64_t n, int64_t* newlen, int32_t* A,
                              RoundCounters* ctr);
__global__ void k_sort_rows_warp(const uint64_t* fse_new, uint32_t* fhub_new, const int32_t* A, const int32_t* U,
                                 int r1_all, RoundCounters* ctr, int32_t* big, int32_t* giant);
// Dynamic shared memory of k_sort_rows_radix: two row buffers of 16,384
// entries and a 32-warp x (256 + 1)-digit histogram.
constexpr int kSortRadixSmemBytes = (2 * 16384 + 257 * 32) * 4;
__global__ void k_sort_rows_radix(const uint64_t* fse_new, uint32_t* fhub_new, const int32_t* big, const int* nbig,
                                  const RoundCounters* ctr);
__global__ void k_sort_rows_block(const uint64_t* fse_new, uint32_t* fhub_new, const int32_t* big, const int* nbig,
                                  uint32_t* scratch, int64_t scratch_words, const RoundCounters* ctr);
__global__ void k_merge_old(const int64_t* loff, const uint32_t* lent, const int64_t* loff_new, uint32_t* lent_new,
                            const uint64_t* fse_new, const uint32_t* fhub_new, int64_t n, const RoundCounters* ctr);
__global__ void k_merge_new(const int64_t* loff, const uint32_t* lent, const int64_t* loff_new, uint32_t* lent_new,
                            const uint64_t* fse_new, const uint32_t* fhub_new, const int32_t* A,
                            const RoundCounters* ctr, uint32_t* top);
__global__ void k_top_init(uint32_t* top, int64_t n);
__global__ void k_final_len(const int64_t* loff, const int32_t* inv, int64_t n, int64_t* len);
__global__ void k_finalize(const int64_t* loff, const uint32_t* lent, const int32_t* inv, const int64_t* out_off,
                           uint32_t* out_packed, uint32_t* out_hub, uint8_t* out_dist, int64_t n,
                           RoundCounters* ctr);

}  // namespace plb
