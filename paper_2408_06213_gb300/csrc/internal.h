// internal.h -- context layout and launcher declarations shared by the brr
// translation units (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/brr.h"

struct brr_ctx {
    int device = 0;
    int num_sms = 0;
    int max_smem_optin = 0;
    int *d_err = nullptr;       // sticky device error word
    int *h_err = nullptr;       // pinned host copy
    // scratch for global-memory shuffles
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    // launch parameters of the staged shuffle kernels, per element size
    // (index 0: 4 bytes, 1: 8 bytes), computed on first use
    bool staged_ready[2] = {false, false};
    uint32_t staged_cap[2] = {0, 0};       // longest array staged in one CTA
    int staged_per_sm[2] = {0, 0};         // resident CTAs per SM
    int staged_clusters[2] = {0, 0};       // resident clusters
    int rounds_per_sm[2] = {0, 0};         // resident CTAs of the rounds kernel
    int long_per_sm[2] = {0, 0};           // resident CTAs of the long-array kernel
    // how shuffles apply their swaps (brr_swap_method)
    uint32_t swap_method = 0;
    // attempts a bulk-dice batch may use before BRR_ERETRY (2^16; lowered
    // only by the brr_selftest_attempt_limit test hook)
    uint32_t attempt_limit = 1u << 16;
    // kernel routing of the chain-resolution shuffles (brr_tune)
    struct {
        uint64_t single_cta_max = 4096;    // one array: one CTA up to this length, else the grid
        uint64_t small_max = 2048;         // batched size classes: small CTAs up to this length,
        uint64_t medium_max = 8192;        //   medium CTAs up to this, then large CTAs
        uint64_t grid_cooperative = 1;     // one array on the grid: one cooperative launch (1)
                                           //   or one launch per pass (0)
        uint64_t fixed_sweep = 1;          // brr_dice_fixed: sweep kernel (1) or tiled kernel (0)
        uint64_t ordered_push = 0;         // CTA chain kernel: barrier between rounds of batch rolls
        uint64_t window_route = 1;         // batched: small and staged large arrays by reservation windows
    } tune;
    // launch parameters of the chain-resolution kernels, per element size
    bool chain_ready[2] = {false, false};
    struct ChainClass {
        uint32_t lo, hi;      // arrays lo < n <= hi
        uint32_t full_cap;    // staged whole up to this length
        uint32_t link_bytes;  // shared memory for heads, bitmap and links of longer arrays
        size_t smem;          // dynamic shared memory per CTA
        int per_sm;           // resident CTAs per SM
    } chain_cls[2][3] = {};   // small, medium, large
    int chain_long_per_sm[2] = {0, 0};
};

namespace brr {

// Grow ctx scratch to at least `bytes` (synchronous; no-op if large enough).
// With `stream` given and being captured into a CUDA graph, growing is not
// possible: BRR_EINVAL (reserve the scratch with brr_reserve first).
brr_status ensure_scratch(brr_ctx *ctx, size_t bytes, cudaStream_t stream = nullptr);

brr_status launch_dice_var(brr_ctx *ctx, const uint32_t *bm1, const uint32_t *off,
                           uint64_t n_batches, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                           cudaStream_t stream, uint32_t source = BRR_WORDS_SPLITMIX64);
brr_status launch_dice_fixed(brr_ctx *ctx, uint32_t bm1, uint32_t k, uint64_t t_full,
                             uint64_t t_last, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                             cudaStream_t stream);
// The same with the words of another source (brr_word_source); thresholds at
// that source's word size, 1 <= k <= 8 for sources other than SplitMix64.
brr_status launch_dice_fixed_src(brr_ctx *ctx, uint32_t source, uint32_t bm1, uint32_t k, uint64_t t_full,
                                 uint64_t t_last, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                                 cudaStream_t stream);
brr_status launch_threshold_test(const uint64_t *B, uint64_t *t, uint64_t n, cudaStream_t stream);
brr_status launch_shuffle(brr_ctx *ctx, void *data, uint64_t n, uint32_t elem_bytes,
                          uint64_t seed, const brr_schedule *sched, uint32_t *j_out,
                          cudaStream_t stream);
brr_status launch_shuffle_batched(brr_ctx *ctx, void *data, const uint64_t *offsets,
                                  uint32_t n_arrays, uint32_t elem_bytes, const uint64_t *seeds,
                                  uint64_t max_len, const brr_schedule *sched,
                                  cudaStream_t stream);
brr_status launch_sample_batched(brr_ctx *ctx, const uint64_t *n, const uint32_t *m,
                                 const uint64_t *seeds, const uint64_t *out_off, uint32_t n_req,
                                 uint32_t max_m, const brr_schedule *sched, uint32_t *out,
                                 cudaStream_t stream, const uint64_t *host_n_single,
                                 uint32_t host_m_single, uint64_t host_seed_single);

size_t shuffle_scratch_size(uint64_t n, bool need_j);
// Shuffles of up to staged_shuffle_cap() elements run staged in shared memory
// (one CTA, or one thread-block cluster).
uint64_t staged_shuffle_cap();
brr_status launch_shuffle_one_staged(brr_ctx *ctx, void *data, uint64_t n, uint32_t elem_bytes,
                                     uint64_t seed, const brr_schedule *sched, uint32_t *j_out,
                                     cudaStream_t stream);
brr_status launch_shuffle_on_scratch(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                                     const brr_schedule *sched, uint32_t *j_out, void *scratch,
                                     int *err, int num_sms, cudaStream_t stream);

// Swap application by chain resolution (chains.cu).
brr_status launch_chains_batched(brr_ctx *ctx, void *data, const uint64_t *offsets, uint32_t n_arrays,
                                 uint32_t elem_bytes, const uint64_t *seeds, uint64_t max_len,
                                 const brr_schedule *sched, cudaStream_t stream,
                                 uint32_t source = BRR_WORDS_SPLITMIX64);
// Reservation windows (windows.cu) for the batched arrays with lo < n <= hi,
// which must stage whole in their class: cls 0 (128-thread CTAs, the small
// class), 3 (256-thread CTAs, four per SM; n <= windows_quarter_cap), 1
// (512-thread CTAs, two per SM; n <= windows_mid_cap), 2 (1024-thread
// CTAs; n <= windows_stage_cap) or 4 (1024-thread CTAs staging only the
// elements, the targets in jt_slots: windows_xl_grid slots of 65,536
// 16-bit entries; n <= windows_xl_cap).  queue: a zeroed work counter;
// list/count: the arrays of the range (null: every array, the others
// skipped); validate: record BRR_EINVAL for invalid arrays.
uint32_t windows_stage_cap(const brr_ctx *ctx, uint32_t elem_bytes);
uint32_t windows_mid_cap(const brr_ctx *ctx, uint32_t elem_bytes);
uint32_t windows_quarter_cap(const brr_ctx *ctx, uint32_t elem_bytes);
uint32_t windows_xl_cap(const brr_ctx *ctx, uint32_t elem_bytes);
uint32_t windows_xl_grid(const brr_ctx *ctx);
brr_status launch_windows_range(brr_ctx *ctx, void *data, const uint64_t *offsets, uint32_t n_arrays,
                                uint32_t elem_bytes, const uint64_t *seeds, uint64_t max_len, const uint64_t *nk,
                                uint32_t k_max, uint32_t cls, uint32_t lo, uint32_t hi, uint32_t *queue,
                                const uint32_t *list, const uint32_t *count, bool validate, cudaStream_t stream,
                                uint32_t source, uint16_t *jt_slots = nullptr);
brr_status launch_chains_one(brr_ctx *ctx, void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                             const brr_schedule *sched, uint32_t *j_out, cudaStream_t stream);
size_t chains_grid_scratch(uint64_t n, uint32_t elem_bytes);
brr_status chains_reserve(brr_ctx *ctx, uint64_t max_len, size_t *bytes);
brr_status launch_chains_grid(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                              const brr_schedule *sched, uint32_t *j_out, void *scratch, int *err,
                              int num_sms, cudaStream_t stream, bool cooperative,
                              const uint32_t *j_in = nullptr);
// Swap-index kernels of a shuffle: the Theorem 1 chain on each word source
// (the values equal brr_word_source) and the naive division method.
enum JgenKind : uint32_t {
    kJgenChain = BRR_WORDS_SPLITMIX64,
    kJgenChaCha20 = BRR_WORDS_CHACHA20,
    kJgenSplitMix32 = BRR_WORDS_SPLITMIX32,
    kJgenNaive = 16
};
brr_status launch_swap_indices(brr_ctx *ctx, uint64_t n, uint64_t seed, const brr_schedule *sched,
                               uint32_t *j_out, uint32_t kind, cudaStream_t stream);
brr_status launch_shuffle_jgen(brr_ctx *ctx, uint32_t kind, void *data, uint64_t n, uint32_t elem_bytes,
                               uint64_t seed, const brr_schedule *sched, uint32_t *j_out,
                               cudaStream_t stream);

inline brr_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return BRR_OK;
    if (e == cudaErrorMemoryAllocation) return BRR_ENOMEM;
    return BRR_ECUDA;
}

}  // namespace brr
