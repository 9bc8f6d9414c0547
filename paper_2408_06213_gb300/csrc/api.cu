// api.cu -- the extern "C" entry points of libbrr: context management,
// host-side validation and planning, and dispatch to the kernel launchers.
#include <cstdio>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "brr_common.cuh"
#include "internal.h"

using brr::u128;

namespace brr {

brr_status ensure_scratch(brr_ctx *ctx, size_t bytes, cudaStream_t stream) {
    if (ctx->scratch_bytes >= bytes) return BRR_OK;
    if (stream) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
            cudaGetLastError();
            return BRR_ECUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) return BRR_EINVAL;  // no allocation while capturing
    }
    // grow geometrically so that a sweep of sizes does not reallocate often
    size_t want = bytes;
    if (want < ctx->scratch_bytes * 3 / 2) want = ctx->scratch_bytes * 3 / 2;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (want == bytes) return BRR_ENOMEM;
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) { cudaGetLastError(); return BRR_ENOMEM; }
        want = bytes;
    }
    if (ctx->scratch) {
        // the old buffer may still be in use by queued work
        cudaDeviceSynchronize();
        cudaFree(ctx->scratch);
    }
    ctx->scratch = p;
    ctx->scratch_bytes = want;
    return BRR_OK;
}

}  // namespace brr

// An NVTX range named after a public call, open while the call queues its
// work (the kernels run asynchronously after it), so that a timeline tool
// (nsys) shows each call beside the kernels it launched.  Without a tool
// attached the push and pop do nothing.
namespace {
struct CallRange {
    explicit CallRange(const char *name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange &) = delete;
    CallRange &operator=(const CallRange &) = delete;
};
}  // namespace

static const brr_schedule *resolve_sched(const brr_schedule *s, brr_schedule *tmp) {
    if (s) return s;
    brr_schedule_paper(tmp);
    return tmp;
}

extern "C" {

void brr_schedule_paper(brr_schedule *s) {
    if (!s) return;
    std::memset(s, 0, sizeof *s);
    s->n_k[2] = 1ull << 30;
    s->n_k[3] = 1ull << 19;
    s->n_k[4] = 1ull << 14;
    s->n_k[5] = 1ull << 11;
    s->n_k[6] = 1ull << 9;
    s->k_max = 6;
}

const char *brr_status_str(brr_status s) {
    switch (s) {
    case BRR_OK: return "BRR_OK";
    case BRR_EINVAL: return "BRR_EINVAL: invalid argument or input";
    case BRR_ENOMEM: return "BRR_ENOMEM: scratch allocation failed";
    case BRR_ECUDA: return "BRR_ECUDA: CUDA runtime error";
    case BRR_ERETRY: return "BRR_ERETRY: batch rejected 2^16 times";
    case BRR_ETIMEOUT: return "BRR_ETIMEOUT: bounded device wait ran out";
    case BRR_ENODEV: return "BRR_ENODEV: no CUDA device";
    }
    return "BRR_?: unknown status";
}

const char *brr_version(void) { return "brr 0.1 (sm_103a)"; }

brr_status brr_shuffle_plan(uint64_t n, uint64_t stop, const brr_schedule *sched,
                            brr_segment *segs, uint32_t max_segs, uint32_t *n_segs,
                            uint64_t *n_batches) {
    brr_schedule tmp;
    sched = resolve_sched(sched, &tmp);
    if (!brr::sched_valid(sched->n_k, sched->k_max)) return BRR_EINVAL;
    if (n > 0xFFFFFFFFull) return BRR_EINVAL;
    if (stop > (n > 1 ? n : 1)) return BRR_EINVAL;
    if (stop == 0) stop = 1;
    brr::Seg tmpsegs[brr::kMaxSegs];
    uint64_t nb = 0;
    const int ns = brr::plan_segments(n, stop, sched->n_k, sched->k_max, tmpsegs, brr::kMaxSegs, &nb);
    if (ns < 0) return BRR_EINVAL;
    for (int s = 0; s < ns && (uint32_t)s < max_segs; s++) {
        segs[s].g0 = tmpsegs[s].g0;
        segs[s].count = tmpsegs[s].count;
        segs[s].u = tmpsegs[s].u;
        segs[s].i0 = tmpsegs[s].i0;
        segs[s].k = tmpsegs[s].k;
    }
    if (n_segs) *n_segs = (uint32_t)ns;
    if (n_batches) *n_batches = nb;
    return BRR_OK;
}

brr_status brr_create(brr_ctx **out) {
    if (!out) return BRR_EINVAL;
    *out = nullptr;
    int dev = 0, count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return BRR_ENODEV;
    }
    if (cudaGetDevice(&dev) != cudaSuccess) return BRR_ENODEV;
    brr_ctx *ctx = new brr_ctx();
    ctx->device = dev;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaError_t e = cudaMalloc(&ctx->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_err, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_err) cudaFree(ctx->d_err);
        delete ctx;
        return BRR_ECUDA;
    }
    *ctx->h_err = 0;
    *out = ctx;
    return BRR_OK;
}

brr_status brr_destroy(brr_ctx *ctx) {
    if (!ctx) return BRR_EINVAL;
    cudaDeviceSynchronize();
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    delete ctx;
    return BRR_OK;
}

brr_status brr_last_device_error(brr_ctx *ctx, brr_stream_t stream) {
    if (!ctx) return BRR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return brr::cuda_status(e);
    return (brr_status)*ctx->h_err;
}

brr_status brr_reserve(brr_ctx *ctx, uint64_t max_shuffle_len, uint64_t max_sample_m) {
    const CallRange range("brr_reserve");
    if (!ctx || max_shuffle_len > 0xFFFFFFFEull) return BRR_EINVAL;
    // reservation rounds, per element: reservation word, two pending-pair
    // lists, swap indices; samples use the same per-slot layout
    const uint64_t elems = max_shuffle_len > 4 * max_sample_m ? max_shuffle_len : 4 * max_sample_m;
    size_t chains = 0;
    const brr_status st = brr::chains_reserve(ctx, max_shuffle_len, &chains);
    if (st != BRR_OK) return st;
    const size_t rounds = (size_t)elems * 24 + (1u << 16);
    return brr::ensure_scratch(ctx, rounds > chains ? rounds : chains);
}

brr_status brr_dice(brr_ctx *ctx, const uint32_t *bm1_dev, const uint32_t *batch_off_dev,
                    uint64_t n_batches, uint64_t n_rolls, uint64_t seed, uint32_t *out_dev,
                    brr_stream_t stream) {
    const CallRange range("brr_dice");
    if (!ctx) return BRR_EINVAL;
    if (n_rolls > 0xFFFFFFFFull || n_batches > 0xFFFFFFC0ull) return BRR_EINVAL;
    if (batch_off_dev == nullptr && n_batches != n_rolls) return BRR_EINVAL;
    if (n_rolls > 0 && (!bm1_dev || !out_dev)) return BRR_EINVAL;
    return brr::launch_dice_var(ctx, bm1_dev, batch_off_dev, n_batches, n_rolls, seed, out_dev,
                                (cudaStream_t)stream);
}

brr_status brr_dice_words(brr_ctx *ctx, uint32_t source, const uint32_t *bm1_dev, const uint32_t *batch_off_dev,
                          uint64_t n_batches, uint64_t n_rolls, uint64_t seed, uint32_t *out_dev,
                          brr_stream_t stream) {
    const CallRange range("brr_dice_words");
    if (source > BRR_WORDS_SPLITMIX32) return BRR_EINVAL;
    if (!ctx) return BRR_EINVAL;
    if (n_rolls > 0xFFFFFFFFull || n_batches > 0xFFFFFFC0ull) return BRR_EINVAL;
    if (batch_off_dev == nullptr && n_batches != n_rolls) return BRR_EINVAL;
    if (n_rolls > 0 && (!bm1_dev || !out_dev)) return BRR_EINVAL;
    return brr::launch_dice_var(ctx, bm1_dev, batch_off_dev, n_batches, n_rolls, seed, out_dev,
                                (cudaStream_t)stream, source);
}

brr_status brr_dice_fixed(brr_ctx *ctx, uint64_t b, uint32_t k, uint64_t n_rolls, uint64_t seed,
                          uint32_t *out_dev, brr_stream_t stream) {
    const CallRange range("brr_dice_fixed");
    if (!ctx || b == 0 || b > (1ull << 32) || k == 0 || k > 64) return BRR_EINVAL;
    if (n_rolls >= (1ull << 40)) return BRR_EINVAL;
    if (n_rolls > 0 && !out_dev) return BRR_EINVAL;
    const u128 W = (u128)1 << 64;
    u128 Bk = 1;
    for (uint32_t i = 0; i < k; i++) {
        Bk *= b;
        if (Bk > W) return BRR_EINVAL;
    }
    const uint64_t t_full = (uint64_t)(W % Bk);
    const uint32_t rem = (uint32_t)(n_rolls % k);
    u128 Br = 1;
    for (uint32_t i = 0; i < rem; i++) Br *= b;
    const uint64_t t_last = rem ? (uint64_t)(W % Br) : t_full;
    return brr::launch_dice_fixed(ctx, (uint32_t)(b - 1), k, t_full, t_last, n_rolls, seed, out_dev,
                                  (cudaStream_t)stream);
}

brr_status brr_dice_fixed_words(brr_ctx *ctx, uint32_t source, uint64_t b, uint32_t k, uint64_t n_rolls,
                                uint64_t seed, uint32_t *out_dev, brr_stream_t stream) {
    const CallRange range("brr_dice_fixed_words");
    if (source == BRR_WORDS_SPLITMIX64) return brr_dice_fixed(ctx, b, k, n_rolls, seed, out_dev, stream);
    if (source != BRR_WORDS_CHACHA20 && source != BRR_WORDS_SPLITMIX32) return BRR_EINVAL;
    if (!ctx || b == 0 || b > (1ull << 32) || k == 0 || k > 8) return BRR_EINVAL;
    if (n_rolls >= (1ull << 40)) return BRR_EINVAL;
    if (n_rolls > 0 && !out_dev) return BRR_EINVAL;
    const u128 W = (u128)1 << (source == BRR_WORDS_SPLITMIX32 ? 32 : 64);
    u128 Bk = 1;
    for (uint32_t i = 0; i < k; i++) {
        Bk *= b;
        if (Bk > W) return BRR_EINVAL;
    }
    const uint64_t t_full = (uint64_t)(W % Bk);
    const uint32_t rem = (uint32_t)(n_rolls % k);
    u128 Br = 1;
    for (uint32_t i = 0; i < rem; i++) Br *= b;
    const uint64_t t_last = rem ? (uint64_t)(W % Br) : t_full;
    return brr::launch_dice_fixed_src(ctx, source, (uint32_t)(b - 1), k, t_full, t_last, n_rolls, seed, out_dev,
                                      (cudaStream_t)stream);
}

brr_status brr_shuffle(brr_ctx *ctx, void *data_dev, uint64_t n, uint32_t elem_bytes,
                       uint64_t seed, const brr_schedule *sched, uint32_t *j_out_dev,
                       brr_stream_t stream) {
    const CallRange range("brr_shuffle");
    brr_schedule tmp;
    sched = resolve_sched(sched, &tmp);
    if (!ctx || (elem_bytes != 4 && elem_bytes != 8) || n > 0xFFFFFFFEull) return BRR_EINVAL;
    if (!brr::sched_valid(sched->n_k, sched->k_max)) return BRR_EINVAL;
    if (n > 1 && !data_dev && !j_out_dev) return BRR_EINVAL;
    if (!data_dev)  // swap indices only
        return brr::launch_swap_indices(ctx, n, seed, sched, j_out_dev, brr::kJgenChain,
                                        (cudaStream_t)stream);
    if (ctx->swap_method == BRR_SWAP_ROUNDS || n <= 1)
        return brr::launch_shuffle(ctx, data_dev, n, elem_bytes, seed, sched, j_out_dev,
                                   (cudaStream_t)stream);
    return brr::launch_chains_one(ctx, data_dev, n, elem_bytes, seed, sched, j_out_dev,
                                  (cudaStream_t)stream);
}

brr_status brr_shuffle_naive(brr_ctx *ctx, void *data_dev, uint64_t n, uint32_t elem_bytes,
                             uint64_t seed, const brr_schedule *sched, uint32_t *j_out_dev,
                             brr_stream_t stream) {
    const CallRange range("brr_shuffle_naive");
    brr_schedule tmp;
    if (!sched) {
        brr_schedule_naive2(&tmp);
        sched = &tmp;
    }
    if (!ctx || (elem_bytes != 4 && elem_bytes != 8) || n > 0xFFFFFFFEull) return BRR_EINVAL;
    if (!brr::sched_valid(sched->n_k, sched->k_max)) return BRR_EINVAL;
    if (n > 1 && !data_dev && !j_out_dev) return BRR_EINVAL;
    if (!data_dev)  // swap indices only
        return brr::launch_swap_indices(ctx, n, seed, sched, j_out_dev, brr::kJgenNaive,
                                        (cudaStream_t)stream);
    return brr::launch_shuffle_jgen(ctx, brr::kJgenNaive, data_dev, n, elem_bytes, seed, sched, j_out_dev,
                                    (cudaStream_t)stream);
}

void brr_schedule_l32(brr_schedule *s) {
    if (!s) return;
    for (int k = 0; k <= BRR_SCHED_KMAX; k++) s->n_k[k] = 0;
    s->n_k[2] = 1ull << 14;
    s->n_k[3] = 1ull << 9;
    s->n_k[4] = 1ull << 6;
    s->k_max = 4;
}

brr_status brr_shuffle_words(brr_ctx *ctx, uint32_t source, void *data_dev, uint64_t n,
                             uint32_t elem_bytes, uint64_t seed, const brr_schedule *sched,
                             uint32_t *j_out_dev, brr_stream_t stream) {
    const CallRange range("brr_shuffle_words");
    if (source == BRR_WORDS_SPLITMIX64)
        return brr_shuffle(ctx, data_dev, n, elem_bytes, seed, sched, j_out_dev, stream);
    if (source != BRR_WORDS_CHACHA20 && source != BRR_WORDS_SPLITMIX32) return BRR_EINVAL;
    brr_schedule tmp;
    if (!sched) {
        if (source == BRR_WORDS_SPLITMIX32)
            brr_schedule_l32(&tmp);
        else
            brr_schedule_paper(&tmp);
        sched = &tmp;
    }
    const uint32_t L = source == BRR_WORDS_SPLITMIX32 ? 32 : 64;
    if (!ctx || (elem_bytes != 4 && elem_bytes != 8) || n > 0xFFFFFFFEull) return BRR_EINVAL;
    if (!brr::sched_valid_bits(sched->n_k, sched->k_max, L)) return BRR_EINVAL;
    if (n > 1 && !data_dev && !j_out_dev) return BRR_EINVAL;
    if (!data_dev)  // swap indices only
        return brr::launch_swap_indices(ctx, n, seed, sched, j_out_dev, source, (cudaStream_t)stream);
    return brr::launch_shuffle_jgen(ctx, source, data_dev, n, elem_bytes, seed, sched, j_out_dev,
                                    (cudaStream_t)stream);
}

void brr_schedule_naive2(brr_schedule *s) {
    if (!s) return;
    for (int k = 0; k <= BRR_SCHED_KMAX; k++) s->n_k[k] = 0;
    s->n_k[2] = 1ull << 32;
    s->k_max = 2;
}

brr_status brr_set_swap_method(brr_ctx *ctx, uint32_t method) {
    if (!ctx || method > BRR_SWAP_CHAINS) return BRR_EINVAL;
    ctx->swap_method = method;
    return BRR_OK;
}

static uint64_t *tune_slot(brr_ctx *ctx, uint32_t param) {
    switch (param) {
        case BRR_TUNE_SINGLE_CTA_MAX: return &ctx->tune.single_cta_max;
        case BRR_TUNE_SMALL_MAX: return &ctx->tune.small_max;
        case BRR_TUNE_MEDIUM_MAX: return &ctx->tune.medium_max;
        case BRR_TUNE_GRID_COOPERATIVE: return &ctx->tune.grid_cooperative;
        case BRR_TUNE_FIXED_SWEEP: return &ctx->tune.fixed_sweep;
        case BRR_TUNE_ORDERED_PUSH: return &ctx->tune.ordered_push;
        case BRR_TUNE_WINDOW_ROUTE: return &ctx->tune.window_route;
        default: return nullptr;
    }
}

brr_status brr_tune(brr_ctx *ctx, uint32_t param, uint64_t value) {
    if (!ctx) return BRR_EINVAL;
    uint64_t *slot = tune_slot(ctx, param);
    if (!slot) return BRR_EINVAL;
    if (param == BRR_TUNE_GRID_COOPERATIVE && value > 1) return BRR_EINVAL;
    if (param == BRR_TUNE_FIXED_SWEEP && value > 1) return BRR_EINVAL;
    if (param == BRR_TUNE_ORDERED_PUSH && value > 1) return BRR_EINVAL;
    if (param == BRR_TUNE_WINDOW_ROUTE && value > 1) return BRR_EINVAL;
    if ((param == BRR_TUNE_SMALL_MAX || param == BRR_TUNE_MEDIUM_MAX) && value > 65536) return BRR_EINVAL;
    *slot = value;
    // size classes are laid out again on the next shuffle
    if (param == BRR_TUNE_SMALL_MAX || param == BRR_TUNE_MEDIUM_MAX)
        ctx->chain_ready[0] = ctx->chain_ready[1] = false;
    return BRR_OK;
}

brr_status brr_tune_get(brr_ctx *ctx, uint32_t param, uint64_t *value) {
    if (!ctx || !value) return BRR_EINVAL;
    uint64_t *slot = tune_slot(ctx, param);
    if (!slot) return BRR_EINVAL;
    *value = *slot;
    return BRR_OK;
}

brr_status brr_shuffle_batched_words(brr_ctx *ctx, uint32_t source, void *data_dev, const uint64_t *offsets_dev,
                                     uint32_t n_arrays, uint32_t elem_bytes, const uint64_t *seeds_dev,
                                     uint64_t max_len, const brr_schedule *sched, brr_stream_t stream) {
    const CallRange range("brr_shuffle_batched_words");
    if (source == BRR_WORDS_SPLITMIX64)
        return brr_shuffle_batched(ctx, data_dev, offsets_dev, n_arrays, elem_bytes, seeds_dev, max_len, sched,
                                   stream);
    if (source != BRR_WORDS_CHACHA20 && source != BRR_WORDS_SPLITMIX32) return BRR_EINVAL;
    brr_schedule tmp;
    if (!sched) {
        if (source == BRR_WORDS_SPLITMIX32)
            brr_schedule_l32(&tmp);
        else
            brr_schedule_paper(&tmp);
        sched = &tmp;
    }
    const uint32_t L = source == BRR_WORDS_SPLITMIX32 ? 32 : 64;
    if (!ctx || (elem_bytes != 4 && elem_bytes != 8) || max_len > 0xFFFFFFFEull) return BRR_EINVAL;
    if (!brr::sched_valid_bits(sched->n_k, sched->k_max, L)) return BRR_EINVAL;
    if (n_arrays == 0) return BRR_OK;
    if (!data_dev || !offsets_dev || !seeds_dev) return BRR_EINVAL;
    return brr::launch_chains_batched(ctx, data_dev, offsets_dev, n_arrays, elem_bytes, seeds_dev, max_len, sched,
                                      (cudaStream_t)stream, source);
}

brr_status brr_shuffle_batched(brr_ctx *ctx, void *data_dev, const uint64_t *offsets_dev,
                               uint32_t n_arrays, uint32_t elem_bytes, const uint64_t *seeds_dev,
                               uint64_t max_len, const brr_schedule *sched, brr_stream_t stream) {
    const CallRange range("brr_shuffle_batched");
    brr_schedule tmp;
    sched = resolve_sched(sched, &tmp);
    if (!ctx || (elem_bytes != 4 && elem_bytes != 8) || max_len > 0xFFFFFFFEull) return BRR_EINVAL;
    if (!brr::sched_valid(sched->n_k, sched->k_max)) return BRR_EINVAL;
    if (n_arrays == 0) return BRR_OK;
    if (!data_dev || !offsets_dev || !seeds_dev) return BRR_EINVAL;
    if (ctx->swap_method == BRR_SWAP_ROUNDS)
        return brr::launch_shuffle_batched(ctx, data_dev, offsets_dev, n_arrays, elem_bytes, seeds_dev,
                                           max_len, sched, (cudaStream_t)stream);
    return brr::launch_chains_batched(ctx, data_dev, offsets_dev, n_arrays, elem_bytes, seeds_dev,
                                      max_len, sched, (cudaStream_t)stream);
}

brr_status brr_sample(brr_ctx *ctx, uint64_t n, uint32_t m, uint64_t seed,
                      const brr_schedule *sched, uint32_t *out_dev, brr_stream_t stream) {
    const CallRange range("brr_sample");
    brr_schedule tmp;
    sched = resolve_sched(sched, &tmp);
    if (!ctx || n > 0xFFFFFFFFull || m > n || m > (1u << 20)) return BRR_EINVAL;
    if (!brr::sched_valid(sched->n_k, sched->k_max)) return BRR_EINVAL;
    if (m == 0) return BRR_OK;
    if (!out_dev) return BRR_EINVAL;
    return brr::launch_sample_batched(ctx, nullptr, nullptr, nullptr, nullptr, 1, m, sched, out_dev,
                                      (cudaStream_t)stream, &n, m, seed);
}

brr_status brr_sample_batched(brr_ctx *ctx, const uint64_t *n_dev, const uint32_t *m_dev,
                              const uint64_t *seeds_dev, const uint64_t *out_off_dev,
                              uint32_t n_req, uint32_t max_m, const brr_schedule *sched,
                              uint32_t *out_dev, brr_stream_t stream) {
    const CallRange range("brr_sample_batched");
    brr_schedule tmp;
    sched = resolve_sched(sched, &tmp);
    if (!ctx || max_m > (1u << 20)) return BRR_EINVAL;
    if (!brr::sched_valid(sched->n_k, sched->k_max)) return BRR_EINVAL;
    if (n_req == 0 || max_m == 0) return BRR_OK;
    if (!n_dev || !m_dev || !seeds_dev || !out_off_dev || !out_dev) return BRR_EINVAL;
    return brr::launch_sample_batched(ctx, n_dev, m_dev, seeds_dev, out_off_dev, n_req, max_m, sched,
                                      out_dev, (cudaStream_t)stream, nullptr, 0, 0);
}

brr_status brr_selftest_attempt_limit(brr_ctx *ctx, uint32_t limit) {
    if (!ctx || limit < 1 || limit > brr::kMaxAttempts) return BRR_EINVAL;
    ctx->attempt_limit = limit;
    return BRR_OK;
}

brr_status brr_selftest_threshold(const uint64_t *B_dev, uint64_t *t_dev, uint64_t n,
                                  brr_stream_t stream) {
    if (n > 0 && (!B_dev || !t_dev)) return BRR_EINVAL;
    return brr::launch_threshold_test(B_dev, t_dev, n, (cudaStream_t)stream);
}

}  // extern "C"
