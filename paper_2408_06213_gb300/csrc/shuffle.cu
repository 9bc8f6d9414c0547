// shuffle.cu -- Fisher-Yates shuffle (Algorithm 1) with batched dice
// (Algorithm 4, Section 6) on the GPU, for arrays in global memory.
//
// Phase 1 (jgen_kernel): one thread per batch of the shuffle plan rolls the
// dice i, i-1, ..., i-k+1 from one word with the Theorem 1 chain and writes
// the swap indices j[i-1-m].  The fast accept test compares the leftover
// word with the segment's upper bound u; only below it is the exact product
// and Lemire threshold formed (Section 5, last paragraphs; Algorithm 4).
//
// Phase 2 (rounds_kernel): the exchanges are applied in deterministic-
// reservation rounds so that the result equals the sequential loop
// "for p = n-1 .. 1: exchange A[p], A[j[p]]".  Every pending swap p reserves
// its two slots with atomicMax(res[slot], p); a swap that holds both slots
// commits (performs the exchange and frees the slots), the others stay
// pending.  A slot is only ever held by the earliest pending swap touching
// it, so a committed swap has no earlier unfinished swap on its slots and
// the committed swaps of a round are disjoint.  The earliest pending swap
// always commits, so the rounds end.  All rounds run in one cooperative
// launch separated by a bounded grid barrier.
#include <algorithm>

#include "brr_common.cuh"
#include "internal.h"
#include "words.cuh"

namespace brr {

constexpr int kJgenThreads = 256;
constexpr int kRoundThreads = 256;
constexpr uint32_t kNoStep = 0xFFFFFFFFu;

struct PlanArgs {
    Seg seg[kMaxSegs];
    int nseg;
    uint64_t n_batches;
};

// Rolls batch g of a plan: writes j[i-1-m] = digit m (die i - m).  Returns
// false if the retry budget ran out.
__device__ __forceinline__ bool roll_shuffle_batch(const Seg *segs, int nseg, uint64_t g,
                                                   uint64_t seed, uint32_t *j) {
    int s = 0;
    while (s + 1 < nseg && segs[s + 1].g0 <= g) s++;
    const Seg sg = segs[s];
    const uint32_t k = sg.k;
    const uint32_t i = sg.i0 - (uint32_t)(g - sg.g0) * k;
    uint32_t a[BRR_SCHED_KMAX];
    uint32_t att = 0;
    uint64_t r = word(seed, g, 0);
#pragma unroll
    for (uint32_t m = 0; m < BRR_SCHED_KMAX; m++)
        if (m < k) a[m] = chain_step(r, i - m);
    bool ok = true;
    if (r < sg.u) {
        const uint64_t B = (uint64_t)falling(i, k);  // exact product, < 2^64
        const uint64_t t = (0 - B) % B;
        while (r < t) {
            if (++att >= kMaxAttempts) { ok = false; break; }
            r = word(seed, g, att);
#pragma unroll
            for (uint32_t m = 0; m < BRR_SCHED_KMAX; m++)
                if (m < k) a[m] = chain_step(r, i - m);
        }
    }
#pragma unroll
    for (uint32_t m = 0; m < BRR_SCHED_KMAX; m++)
        if (m < k) j[i - 1 - m] = a[m];
    return ok;
}

__global__ void __launch_bounds__(kJgenThreads)
jgen_kernel(PlanArgs plan, uint64_t seed, uint32_t *__restrict__ j, int *err) {
    bool ok = true;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < plan.n_batches; g += stride)
        ok = roll_shuffle_batch(plan.seg, plan.nseg, g, seed, j) && ok;
    if (!ok) record_error(err, BRR_ERETRY);
    if (blockIdx.x == 0 && threadIdx.x == 0) j[0] = 0;
}

// The naive batched method (the paper's comparison, Section 3 and its
// appendix listing): the k dice of batch g come from one Lemire roll of their
// product B = i (i-1) ... (i-k+1), split by remainders of successive
// quotients, least significant first: die i - m gets v mod (i - m), then
// v <- v div (i - m).  The threshold 2^64 mod B and the digits use the
// hardware's 64-bit division, as the method prescribes.
__device__ __forceinline__ bool naive_batch(const Seg *segs, int nseg, uint64_t g, uint64_t seed,
                                            uint32_t *j) {
    int s = 0;
    while (s + 1 < nseg && segs[s + 1].g0 <= g) s++;
    const Seg sg = segs[s];
    const uint32_t k = sg.k;
    const uint32_t i = sg.i0 - (uint32_t)(g - sg.g0) * k;
    const uint64_t B = (uint64_t)falling(i, k);  // < 2^64: a product of consecutive integers
    uint32_t att = 0;
    bool ok = true;
    uint64_t r = word(seed, g, 0);
    uint64_t v = __umul64hi(B, r), lo = B * r;
    if (lo < B) {
        const uint64_t t = (0 - B) % B;
        while (lo < t) {
            if (++att >= kMaxAttempts) { ok = false; break; }
            r = word(seed, g, att);
            v = __umul64hi(B, r);
            lo = B * r;
        }
    }
    for (uint32_t m = 0; m < k; m++) {
        const uint32_t b = i - m;
        j[i - 1 - m] = (uint32_t)(v % b);
        v /= b;
    }
    return ok;
}

__global__ void __launch_bounds__(kJgenThreads)
naive_jgen_kernel(PlanArgs plan, uint64_t seed, uint32_t *__restrict__ j, int *err) {
    bool ok = true;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < plan.n_batches; g += stride)
        ok = naive_batch(plan.seg, plan.nseg, g, seed, j) && ok;
    if (!ok) record_error(err, BRR_ERETRY);
    if (blockIdx.x == 0 && threadIdx.x == 0) j[0] = 0;
}

template <uint32_t SRC>
__global__ void __launch_bounds__(kJgenThreads)
words_jgen_kernel(PlanArgs plan, uint64_t seed, uint32_t *__restrict__ j, int *err) {
    bool ok = true;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < plan.n_batches; g += stride)
        ok = roll_plan_batch_src<SRC>(plan.seg, plan.nseg, g, seed, [&](uint32_t pos, uint32_t v) { j[pos] = v; }) &&
             ok;
    if (!ok) record_error(err, BRR_ERETRY);
    if (blockIdx.x == 0 && threadIdx.x == 0) j[0] = 0;
}

// Queues the swap-index kernel of `kind` over a plan.
static cudaError_t launch_jgen(uint32_t kind, const PlanArgs &plan, unsigned grid, uint64_t seed,
                               uint32_t *j, int *err, cudaStream_t stream) {
    switch (kind) {
    case kJgenNaive:
        naive_jgen_kernel<<<grid, kJgenThreads, 0, stream>>>(plan, seed, j, err);
        break;
    case kJgenChaCha20:
        words_jgen_kernel<BRR_WORDS_CHACHA20><<<grid, kJgenThreads, 0, stream>>>(plan, seed, j, err);
        break;
    case kJgenSplitMix32:
        words_jgen_kernel<BRR_WORDS_SPLITMIX32><<<grid, kJgenThreads, 0, stream>>>(plan, seed, j, err);
        break;
    default:
        jgen_kernel<<<grid, kJgenThreads, 0, stream>>>(plan, seed, j, err);
        break;
    }
    return cudaGetLastError();
}

// Warp-aggregated append of (x, j) pairs to a global pending list.
__device__ __forceinline__ void warp_append_pair(bool flag, uint32_t x, uint32_t jx, uint2 *list,
                                                 uint32_t *cnt) {
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(cnt, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) __stcg(&list[base + __popc(mask & ((1u << lane) - 1))], make_uint2(x, jx));
}

template <typename T>
__device__ __forceinline__ void swap_cg(T *A, uint32_t x, uint32_t y) {
    const T a = __ldcg(&A[x]);
    const T b = __ldcg(&A[y]);
    __stcg(&A[x], b);
    __stcg(&A[y], a);
}

struct RoundsArgs {
    void *A;
    const uint32_t *j;     // swap target of every position (kNoStep: no step)
    uint32_t *res;         // reservation word per slot, all zero on entry
    uint2 *list[2];        // pending (x, j[x]) pairs
    uint32_t *cnt;         // [3] rotating pending counters, zero on entry
    uint32_t *bar;         // [2] grid barrier, zero on entry
    uint32_t *rounds_out;  // [1] number of rounds used
    uint32_t x_lo, x_hi;   // round 0 covers positions x_lo .. x_hi - 1
    int *err;
};

// Priority of the swap at position x is x itself (x >= 1): later positions
// are earlier in the sequential order p = n-1, ..., 1.
//
// The pending set shrinks by about a quarter per round, so the last rounds
// hold few swaps; once at most kSoloPending remain, block 0 finishes alone
// with block barriers instead of grid barriers (the other blocks leave).
constexpr uint32_t kSoloPending = 2048;

template <typename T>
__global__ void __launch_bounds__(kRoundThreads) rounds_kernel(RoundsArgs args) {
    T *A = static_cast<T *>(args.A);
    const uint32_t tid = threadIdx.x;
    uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t gbase = (uint64_t)blockIdx.x * blockDim.x;
    uint64_t count = args.x_hi - args.x_lo;
    bool solo = gridDim.x == 1;
    uint32_t round = 0;
    for (;;) {
        // every round commits the earliest pending swap: more rounds than
        // positions means corrupted state, reported instead of looping
        if ((uint64_t)round > (uint64_t)(args.x_hi - args.x_lo) + 1) {
            if (blockIdx.x == 0 && tid == 0) record_error(args.err, BRR_ETIMEOUT);
            return;
        }
        const uint2 *cur = (round & 1) ? args.list[1] : args.list[0];
        // ---- reserve
        for (uint64_t base = gbase; base < count; base += gstride) {
            const uint64_t idx = base + tid;
            if (idx >= count) break;
            uint32_t x, jx;
            if (round == 0) {
                x = args.x_hi - 1 - (uint32_t)idx;
                jx = args.j[x];
            } else {
                const uint2 e = __ldcg(&cur[idx]);
                x = e.x;
                jx = e.y;
            }
            if (jx == kNoStep) continue;
            atomicMax(&args.res[x], x);
            if (jx != x) atomicMax(&args.res[jx], x);
        }
        if (solo) __syncthreads();
        else if (!grid_barrier(args.bar, args.err)) return;
        // ---- commit or stay pending
        uint2 *next = (round & 1) ? args.list[0] : args.list[1];
        uint32_t *next_cnt = &args.cnt[(round + 1) % 3];
        for (uint64_t base = gbase; base < count; base += gstride) {
            const uint64_t idx = base + tid;
            bool pend = false;
            uint32_t x = 0, jx = kNoStep;
            if (idx < count) {
                if (round == 0) {
                    x = args.x_hi - 1 - (uint32_t)idx;
                    jx = args.j[x];
                } else {
                    const uint2 e = __ldcg(&cur[idx]);
                    x = e.x;
                    jx = e.y;
                }
                if (jx != kNoStep) {
                    if (__ldcg(&args.res[x]) == x && __ldcg(&args.res[jx]) == x) {
                        if (jx != x) swap_cg(A, x, jx);
                        __stcg(&args.res[x], 0u);
                        __stcg(&args.res[jx], 0u);
                    } else {
                        pend = true;
                    }
                }
            }
            warp_append_pair(pend, x, jx, next, next_cnt);
        }
        if (blockIdx.x == 0 && tid == 0) args.cnt[(round + 2) % 3] = 0;
        if (solo) __syncthreads();
        else if (!grid_barrier(args.bar, args.err)) return;
        count = *(volatile uint32_t *)next_cnt;
        round++;
        if (count == 0) break;
        if (!solo && count <= kSoloPending) {
            // every block read the same count: all but block 0 leave together
            if (blockIdx.x != 0) return;
            solo = true;
            gstride = blockDim.x;
            gbase = 0;
        }
    }
    if (blockIdx.x == 0 && tid == 0) *args.rounds_out = round;
}

// Scratch layout for a global-memory shuffle of n positions.
struct ShuffleScratch {
    uint32_t *res;
    uint2 *list0, *list1;
    uint32_t *jbuf;
    uint32_t *ctrl;  // cnt[3], bar[2], rounds[1]
};

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static size_t shuffle_scratch_bytes(uint64_t n, bool need_j) {
    size_t b = 0;
    b += align_up(n * sizeof(uint32_t), 256);
    b += 2 * align_up(n * sizeof(uint2), 256);
    if (need_j) b += align_up(n * sizeof(uint32_t), 256);
    b += 256;
    return b;
}

static ShuffleScratch carve(void *base, uint64_t n, bool need_j) {
    ShuffleScratch s;
    char *p = static_cast<char *>(base);
    s.res = reinterpret_cast<uint32_t *>(p);
    p += align_up(n * sizeof(uint32_t), 256);
    s.list0 = reinterpret_cast<uint2 *>(p);
    p += align_up(n * sizeof(uint2), 256);
    s.list1 = reinterpret_cast<uint2 *>(p);
    p += align_up(n * sizeof(uint2), 256);
    s.jbuf = nullptr;
    if (need_j) {
        s.jbuf = reinterpret_cast<uint32_t *>(p);
        p += align_up(n * sizeof(uint32_t), 256);
    }
    s.ctrl = reinterpret_cast<uint32_t *>(p);
    return s;
}

template <typename T>
static brr_status launch_rounds(brr_ctx *ctx, void *A, const uint32_t *j, const ShuffleScratch &s,
                                uint32_t x_lo, uint32_t x_hi, cudaStream_t stream) {
    RoundsArgs args;
    args.A = A;
    args.j = j;
    args.res = s.res;
    args.list[0] = s.list0;
    args.list[1] = s.list1;
    args.cnt = s.ctrl;
    args.bar = s.ctrl + 4;
    args.rounds_out = s.ctrl + 6;
    args.x_lo = x_lo;
    args.x_hi = x_hi;
    args.err = ctx->d_err;
    const void *kern = (const void *)rounds_kernel<T>;
    int &per_sm = ctx->rounds_per_sm[sizeof(T) == 4 ? 0 : 1];
    if (per_sm < 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRoundThreads, 0);
    if (per_sm < 1) return BRR_ECUDA;
    const uint64_t max_blocks = (uint64_t)per_sm * ctx->num_sms;
    // about 16 positions per thread in round 0: fewer blocks make each grid
    // barrier cheaper for small arrays
    const uint64_t want = ((uint64_t)(x_hi - x_lo) + kRoundThreads * 16 - 1) / (kRoundThreads * 16);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, max_blocks));
    void *params[] = {&args};
    return cuda_status(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kRoundThreads), params, 0, stream));
}

brr_status launch_shuffle(brr_ctx *ctx, void *data, uint64_t n, uint32_t elem_bytes,
                          uint64_t seed, const brr_schedule *sched, uint32_t *j_out,
                          cudaStream_t stream) {
    if (n <= 1) {
        if (n == 1 && j_out) return cuda_status(cudaMemsetAsync(j_out, 0, sizeof(uint32_t), stream));
        return BRR_OK;
    }
    // arrays that fit one CTA's or one cluster's shared memory run staged there
    if (n <= staged_shuffle_cap())
        return launch_shuffle_one_staged(ctx, data, n, elem_bytes, seed, sched, j_out, stream);
    PlanArgs plan;
    plan.nseg = plan_segments(n, 1, sched->n_k, sched->k_max, plan.seg, kMaxSegs, &plan.n_batches);
    if (plan.nseg < 0) return BRR_EINVAL;
    const bool need_j = j_out == nullptr;
    brr_status st = ensure_scratch(ctx, shuffle_scratch_bytes(n, need_j), stream);
    if (st != BRR_OK) return st;
    ShuffleScratch s = carve(ctx->scratch, n, need_j);
    uint32_t *j = need_j ? s.jbuf : j_out;
    cudaError_t e = cudaMemsetAsync(s.res, 0, n * sizeof(uint32_t), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.ctrl, 0, 8 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_status(e);
    const uint64_t want = (plan.n_batches + kJgenThreads - 1) / kJgenThreads;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)ctx->num_sms * 8));
    jgen_kernel<<<grid, kJgenThreads, 0, stream>>>(plan, seed, j, ctx->d_err);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    if (elem_bytes == 4)
        return launch_rounds<uint32_t>(ctx, data, j, s, 1, (uint32_t)n, stream);
    return launch_rounds<uint64_t>(ctx, data, j, s, 1, (uint32_t)n, stream);
}

// Only the swap indices of a shuffle (data == nullptr): one thread per batch,
// with the kernel of `kind` (the Theorem 1 chain on one of the word sources,
// or the naive division method).
brr_status launch_swap_indices(brr_ctx *ctx, uint64_t n, uint64_t seed, const brr_schedule *sched,
                               uint32_t *j_out, uint32_t kind, cudaStream_t stream) {
    if (n == 0) return BRR_OK;
    if (n == 1) return cuda_status(cudaMemsetAsync(j_out, 0, sizeof(uint32_t), stream));
    PlanArgs plan;
    plan.nseg = plan_segments(n, 1, sched->n_k, sched->k_max, plan.seg, kMaxSegs, &plan.n_batches);
    if (plan.nseg < 0) return BRR_EINVAL;
    const uint64_t want = (plan.n_batches + kJgenThreads - 1) / kJgenThreads;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)ctx->num_sms * 8));
    return cuda_status(launch_jgen(kind, plan, grid, seed, j_out, ctx->d_err, stream));
}

// A shuffle whose swap indices come from a separate kernel of `kind` (the
// naive batched method, or another word source), applied by the context's
// swap method (chain resolution on the grid, or rounds).
brr_status launch_shuffle_jgen(brr_ctx *ctx, uint32_t kind, void *data, uint64_t n, uint32_t elem_bytes,
                               uint64_t seed, const brr_schedule *sched, uint32_t *j_out,
                               cudaStream_t stream) {
    if (n <= 1) {
        if (n == 1 && j_out) return cuda_status(cudaMemsetAsync(j_out, 0, sizeof(uint32_t), stream));
        return BRR_OK;
    }
    PlanArgs plan;
    plan.nseg = plan_segments(n, 1, sched->n_k, sched->k_max, plan.seg, kMaxSegs, &plan.n_batches);
    if (plan.nseg < 0) return BRR_EINVAL;
    const uint64_t want = (plan.n_batches + kJgenThreads - 1) / kJgenThreads;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)ctx->num_sms * 8));
    const bool need_j = j_out == nullptr;
    cudaError_t e;
    if (ctx->swap_method == BRR_SWAP_ROUNDS) {
        brr_status st = ensure_scratch(ctx, shuffle_scratch_bytes(n, need_j), stream);
        if (st != BRR_OK) return st;
        ShuffleScratch s = carve(ctx->scratch, n, need_j);
        uint32_t *j = need_j ? s.jbuf : j_out;
        e = cudaMemsetAsync(s.res, 0, n * sizeof(uint32_t), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(s.ctrl, 0, 8 * sizeof(uint32_t), stream);
        if (e != cudaSuccess) return cuda_status(e);
        if ((e = launch_jgen(kind, plan, grid, seed, j, ctx->d_err, stream)) != cudaSuccess) return cuda_status(e);
        if (elem_bytes == 4)
            return launch_rounds<uint32_t>(ctx, data, j, s, 1, (uint32_t)n, stream);
        return launch_rounds<uint64_t>(ctx, data, j, s, 1, (uint32_t)n, stream);
    }
    const size_t grid_bytes = align_up(chains_grid_scratch(n, elem_bytes), 256);
    brr_status st = ensure_scratch(ctx, grid_bytes + (need_j ? align_up(n * sizeof(uint32_t), 256) : 0), stream);
    if (st != BRR_OK) return st;
    uint32_t *j = need_j ? reinterpret_cast<uint32_t *>(static_cast<char *>(ctx->scratch) + grid_bytes) : j_out;
    if ((e = launch_jgen(kind, plan, grid, seed, j, ctx->d_err, stream)) != cudaSuccess) return cuda_status(e);
    return launch_chains_grid(data, n, elem_bytes, seed, sched, nullptr, ctx->scratch, ctx->d_err, ctx->num_sms,
                              stream, ctx->tune.grid_cooperative != 0, j);
}

}  // namespace brr

// ------------------------------------------------ caller-provided scratch --
// The same shuffle with scratch and error word supplied by the caller instead
// of a context (used by the entry point that allocates nothing).

namespace brr {

size_t shuffle_scratch_size(uint64_t n, bool need_j) { return shuffle_scratch_bytes(n, need_j); }

template <typename T>
static brr_status launch_rounds_raw(int num_sms, int *err, void *A, const uint32_t *j,
                                    const ShuffleScratch &s, uint32_t x_lo, uint32_t x_hi,
                                    cudaStream_t stream) {
    RoundsArgs args;
    args.A = A;
    args.j = j;
    args.res = s.res;
    args.list[0] = s.list0;
    args.list[1] = s.list1;
    args.cnt = s.ctrl;
    args.bar = s.ctrl + 4;
    args.rounds_out = s.ctrl + 6;
    args.x_lo = x_lo;
    args.x_hi = x_hi;
    args.err = err;
    const void *kern = (const void *)rounds_kernel<T>;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRoundThreads, 0);
    if (per_sm < 1) return BRR_ECUDA;
    const uint64_t max_blocks = (uint64_t)per_sm * num_sms;
    const uint64_t want = ((uint64_t)(x_hi - x_lo) + kRoundThreads * 16 - 1) / (kRoundThreads * 16);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, max_blocks));
    void *params[] = {&args};
    return cuda_status(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kRoundThreads), params, 0, stream));
}

brr_status launch_shuffle_on_scratch(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                                     const brr_schedule *sched, uint32_t *j_out, void *scratch,
                                     int *err, int num_sms, cudaStream_t stream) {
    if (n <= 1) {
        if (n == 1 && j_out) return cuda_status(cudaMemsetAsync(j_out, 0, sizeof(uint32_t), stream));
        return BRR_OK;
    }
    PlanArgs plan;
    plan.nseg = plan_segments(n, 1, sched->n_k, sched->k_max, plan.seg, kMaxSegs, &plan.n_batches);
    if (plan.nseg < 0) return BRR_EINVAL;
    const bool need_j = j_out == nullptr;
    ShuffleScratch s = carve(scratch, n, need_j);
    uint32_t *j = need_j ? s.jbuf : j_out;
    cudaError_t e = cudaMemsetAsync(s.res, 0, n * sizeof(uint32_t), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.ctrl, 0, 8 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_status(e);
    const uint64_t want = (plan.n_batches + kJgenThreads - 1) / kJgenThreads;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms * 8));
    jgen_kernel<<<grid, kJgenThreads, 0, stream>>>(plan, seed, j, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    if (elem_bytes == 4)
        return launch_rounds_raw<uint32_t>(num_sms, err, data, j, s, 1, (uint32_t)n, stream);
    return launch_rounds_raw<uint64_t>(num_sms, err, data, j, s, 1, (uint32_t)n, stream);
}

}  // namespace brr
